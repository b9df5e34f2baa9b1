"""Host model of the barrier protocol of the shared-memory permutation form
(csrc/tc_perm_smem.cu): the A producer, the MMA issuer and the 8 gathering
epilogue warps of a CTA pair, with their stage ring (kSStages slots), the
two TMEM accumulators and the segment structure, run as a discrete-event
simulation over many segment shapes.

It checks what a GPU run cannot show safely: no deadlock, no barrier
phase receiving more arrivals than its count, and no parity wait issued
by a waiter two phases ahead (where the parity of the awaited phase equals
the current one and the wait would pass early).  The variant that deals
stages round-robin to 8 warps over the 5-slot ring is kept as a negative
case: it aliases, which is why the kernel has every warp gather every
stage in order.
"""
import pytest

S = 5           # ring slots (kSStages)
WARPS = 8       # gathering epilogue warps per CTA (kPEpiWarps)


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


def simulate(segs, nkb, round_robin=False):
    """segs: passes per segment; nkb: stages per pass.  Returns normally
    when every role finishes; raises AssertionError on a protocol fault."""
    gathering = 1 if round_robin else WARPS
    full = [Bar(1 + 2 * gathering, f"full{i}") for i in range(S)]
    empty = [Bar(1, f"empty{i}") for i in range(S)]
    tfull = [Bar(1, f"tfull{i}") for i in range(2)]
    tempty = [Bar(2 * WARPS, f"tempty{i}") for i in range(2)]

    def producer():
        sg = 0
        for nps in segs:
            for _ in range((nps + 1) * nkb):
                yield ("w", empty[sg % S], sg // S)
                yield ("a", full[sg % S], 1)   # even CTA's arm + A bytes
                sg += 1

    def mma():
        sg = npass = 0
        for nps in segs:
            for _ in range(-1, nps):
                acc = npass % 2
                yield ("w", tempty[acc], npass // 2)
                for _ in range(nkb):
                    yield ("w", full[sg % S], sg // S + 1)
                    yield ("a", empty[sg % S], 1)
                    sg += 1
                yield ("a", tfull[acc], 1)
                npass += 1

    def worker(e):
        sig0 = npass = 0
        for nps in segs:
            nst = (nps + 1) * nkb
            sl = ((e - sig0 % WARPS) % WARPS) if round_robin else 0
            step = WARPS if round_robin else 1
            for pi in range(-1, nps + 1):
                while pi < nps and sl < (pi + 2) * nkb:
                    sg = sig0 + sl
                    yield ("w", empty[sg % S], sg // S)
                    yield ("a", full[sg % S], 2)   # this warp in both CTAs
                    sl += step
                if pi < 0:
                    continue
                acc = npass % 2
                yield ("w", tfull[acc], npass // 2 + 1)
                yield ("a", tempty[acc], 2)
                npass += 1
            sig0 += nst

    gens = [producer(), mma()] + [worker(e) for e in range(WARPS)]
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


SHAPES = [[1], [3], [1, 1, 1], [3, 1, 5], [8, 2], [17, 4, 9, 1], [60]]


@pytest.mark.parametrize("nkb", [2, 4, 6, 8])
@pytest.mark.parametrize("segs", SHAPES)
def test_protocol_runs_to_completion(segs, nkb):
    simulate(segs, nkb)


def test_round_robin_variant_aliases():
    with pytest.raises(AssertionError) as ex:
        for nkb in (2, 8):
            for segs in SHAPES:
                simulate(segs, nkb, round_robin=True)
    assert ex.value.args[0][0] in ("alias", "overflow")
