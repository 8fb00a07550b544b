"""Host model of the 16-byte input staging of the one-thread-per-half chain kernel
(csrc/tv_flat.cuh, VEC): every asynchronous copy it issues must lie inside its own chain,
start on a 16-byte boundary, and cover every step the lane reads.

A warp holds 16 chains; lane l < 16 runs the left half of chain 16*w + l (nodes 0..mid-1,
mid = n/2), lane l + 16 the right half (nodes n-1..mid+1). Step t of a half is staged in
the 4-step chunk t & ~3: a left half copies nodes t..t+3, a right half nodes n-4-t..n-1-t.
With per-edge weights a right half's step s reads edge n-2-s, found where step s+1's node
is, so right halves stage through step cnt; an empty half (a padding lane of the last
warp, or a chain of no nodes) stages nothing. The staged range of a round ends on a
4-step boundary, at most the half count rounded up (one step more with weights)."""
import pytest

HW, WARP = 16, 32


def staging_plan(nc, n, has_w, empty_rule=True):
    """(warp, lane, chain start, chain length, [(node index, 'y' or 'w')]) of every copy,
    and the steps each lane reads, for a uniform batch of nc chains of n nodes."""
    warps = (nc + HW - 1) // HW
    for wg in range(warps):
        cnts = []
        for lane in range(WARP):
            k = wg * HW + (lane & (HW - 1))
            nn = n if k < nc else 0
            mid = nn >> 1
            cnts.append(0 if nn == 0 else (mid if lane < HW else nn - 1 - mid))
        cmax = max(cnts)
        cmaxs = (cmax + (4 if has_w else 3)) & ~3
        for lane in range(WARP):
            k = wg * HW + (lane & (HW - 1))
            left = lane < HW
            nn = n if k < nc else 0
            start = k * n if k < nc else 0
            cnt = cnts[lane]
            wlag = 1 if (has_w and not left) else 0
            cnt_st = cnt + wlag if (cnt > 0 or not empty_rule) else 0
            copies = []
            for t in range(0, cmaxs, 4):
                if t < cnt_st:
                    copies.append((start + t if left else start + nn - 4 - t, "y"))
                    if has_w:
                        copies.append((start + t if left else start + nn - 4 - t, "w"))
            # steps read: node input of step j, and the weight of step j (+1 on the right)
            reads = [(j, "y") for j in range(cnt)]
            if has_w:
                reads += [(j + wlag, "w") for j in range(cnt)]
            yield wg, lane, start, nn, copies, reads


def violations(nc, n, has_w, empty_rule=True):
    """Copies outside their chain or off the 16-byte grid, and reads of unstaged steps."""
    out = []
    for wg, lane, start, nn, copies, reads in staging_plan(nc, n, has_w, empty_rule):
        for a, _ in copies:
            if a % 4 or a < start or a + 4 > start + nn or a < 0 or a + 4 > nc * n:
                out.append(("copy", wg, lane, a))
        left = lane < HW
        chunks = {(a - start if left else start + nn - 4 - a, arr) for a, arr in copies}
        for s, arr in reads:
            if (s & ~3, arr) not in chunks:
                out.append(("read", wg, lane, s, arr))
    return out


@pytest.mark.parametrize("has_w", [False, True])
@pytest.mark.parametrize("n", [4, 8, 12, 64, 68, 72, 100, 132, 260, 1024])
@pytest.mark.parametrize("nc", [1, 15, 16, 17, 40, 96])
def test_every_staging_copy_stays_in_its_chain(nc, n, has_w):
    assert violations(nc, n, has_w) == []


def test_the_model_catches_an_empty_half_that_stages():
    """Without the empty-half rule each padding lane's right half (no nodes, start 0)
    would copy nodes -4..-1 of y and of w: 8 such lanes in a batch of 40 chains (3 warps)."""
    bad = violations(40, 64, True, empty_rule=False)
    assert len(bad) == 16 and all(v[0] == "copy" and v[3] == -4 for v in bad)
    assert sorted({v[2] for v in bad}) == list(range(24, 32))
    assert violations(40, 64, True) == []
