"""Host model of the barrier protocol of the transposed permutation form
(csrc/tc_perm_mn.cu), run as a discrete-event simulation over many segment
shapes, ring depths and stages per pass.  Per CTA pair it has:
  - in each CTA, the A loader and stage forwarder (warp 0);
  - the even CTA's MMA issuer;
  - in each CTA, the two copying warps;
  - in each CTA, the 8 epilogue warps.
They share the B ring (full on the even CTA; empty and the copies' own
barrier in each CTA), the resident A tiles (afull on the even CTA, aempty in
each CTA) and the two TMEM accumulators.

It checks what a GPU run cannot show safely: no deadlock, no barrier phase
receiving more arrivals than its count, and no parity wait issued by a
waiter two phases ahead (the awaited phase's parity equal to the current
one, so that the wait would pass early).
"""
import pytest

EPI = 8     # epilogue warps per CTA (kPEpiWarps)
COPY = 2    # copying warps per CTA; each warp's 32 threads arrive


class Bar:
    def __init__(self, count, name):
        self.n, self.a, self.ph, self.name = count, 0, 0, name

    def arrive(self, k=1):
        self.a += k
        if self.a > self.n:
            raise AssertionError(("overflow", self.name))
        if self.a == self.n:
            self.ph, self.a = self.ph + 1, 0

    def ready(self, k):
        """A parity wait for 'k phases completed' (parity of phase k - 1)."""
        if (self.ph & 1) == (k & 1) and self.ph < k:
            raise AssertionError(("alias", self.name))
        return self.ph >= k


def simulate(segs, nkb, S, drop_forward=False):
    """segs: passes per segment (each segment adds one r_obs pass); nkb: B
    stages per pass; S: ring slots.  Returns when every role finishes;
    raises AssertionError on a protocol fault.  drop_forward plants a
    mistake: the odd CTA forwards no stage."""
    full = [Bar(2, f"full{i}") for i in range(S)]            # even CTA
    empty = [[Bar(1, f"empty{c}.{i}") for i in range(S)] for c in (0, 1)]
    bfull = [[Bar(32 * COPY, f"bfull{c}.{i}") for i in range(S)]
             for c in (0, 1)]
    tfull = [[Bar(1, f"tfull{c}.{a}") for a in (0, 1)] for c in (0, 1)]
    tempty = [Bar(2 * EPI, f"tempty{a}") for a in (0, 1)]    # even CTA
    # even CTA: its producer's arm (1 arrival) plus both CTAs' A bytes,
    # modelled as one completion per CTA
    afull = Bar(3, "afull")
    aempty = [Bar(1, f"aempty{c}") for c in (0, 1)]

    def loader(c):
        sg = 0
        for seg, nps in enumerate(segs):
            yield ("w", aempty[c], seg)       # parity aph ^ 1: seg phases
            if c == 0:
                yield ("a", afull, 1)         # arm
            yield ("a", afull, 1)             # this CTA's A bytes land
            for _ in range((nps + 1) * nkb):
                yield ("w", bfull[c][sg % S], sg // S + 1)
                if not (drop_forward and c == 1):
                    yield ("a", full[sg % S], 1)  # forward to the even CTA
                sg += 1

    def mma():
        sg = npass = 0
        for seg, nps in enumerate(segs):
            yield ("w", afull, seg + 1)
            for _ in range(-1, nps):
                acc = npass % 2
                yield ("w", tempty[acc], npass // 2)
                for _ in range(nkb):
                    yield ("w", full[sg % S], sg // S + 1)
                    yield ("a", empty[0][sg % S], 1)   # commit, both CTAs
                    yield ("a", empty[1][sg % S], 1)
                    sg += 1
                yield ("a", tfull[0][acc], 1)
                yield ("a", tfull[1][acc], 1)
                npass += 1
            yield ("a", aempty[0], 1)
            yield ("a", aempty[1], 1)

    def copier(c):
        sg = 0
        for nps in segs:
            for _ in range((nps + 1) * nkb):
                yield ("w", empty[c][sg % S], sg // S)
                yield ("a", bfull[c][sg % S], 32)     # the warp's threads
                sg += 1

    def epilogue(c):
        npass = 0
        for nps in segs:
            for _ in range(-1, nps):
                acc = npass % 2
                yield ("w", tfull[c][acc], npass // 2 + 1)
                yield ("a", tempty[acc], 1)
                npass += 1

    gens = [loader(0), loader(1), mma()]
    gens += [copier(c) for c in (0, 1) for _ in range(COPY)]
    gens += [epilogue(c) for c in (0, 1) for _ in range(EPI)]
    cur = [next(g, None) for g in gens]
    while any(c is not None for c in cur):
        moved = False
        for i, c in enumerate(cur):
            while c is not None:
                if c[0] == "w" and not c[1].ready(c[2]):
                    break
                if c[0] == "a":
                    c[1].arrive(c[2])
                c = next(gens[i], None)
                moved = True
            cur[i] = c
        if not moved:
            raise AssertionError(("deadlock",))


SHAPES = [[0], [1], [3], [1, 1, 1], [3, 1, 5], [8, 2], [17, 4, 9, 1], [60]]


@pytest.mark.parametrize("S,nkb", [(3, 1), (3, 2), (3, 3), (3, 4),
                                   (6, 2), (6, 4), (6, 6), (6, 8)])
@pytest.mark.parametrize("segs", SHAPES)
def test_protocol_runs_to_completion(segs, nkb, S):
    simulate(segs, nkb, S)


def test_model_catches_a_missing_forward():
    """A planted mistake (the odd CTA forwards no stage) leaves the even
    CTA's full barriers one arrival short: the model deadlocks, where the
    kernel's bounded waits would report a timeout."""
    with pytest.raises(AssertionError) as ex:
        simulate([3], 2, 3, drop_forward=True)
    assert ex.value.args[0][0] == "deadlock"


def test_model_flags_a_waiter_two_phases_ahead():
    """A waiter two phases ahead of a barrier (awaiting the 4th phase while
    2 have completed) would see the parity it waits for and pass early:
    the model reports it instead of letting it pass."""
    bar = Bar(1, "b")
    bar.arrive()
    bar.arrive()
    with pytest.raises(AssertionError):
        bar.ready(4)
