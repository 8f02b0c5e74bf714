"""Host-side model of the line pass's shared-memory index arithmetic (pat_line.cuh), no GPU.

The kernel writes every exchange-buffer address as a per-thread base plus a compile-time offset,
resolving the bank swizzle per thread.  This test restates, for the CTA shape of every instantiated
line length, (a) the thread -> (line, row, pair half) mapping, (b) the generic swizzle (bit 0 of a row
flipped by bit 0 of row / B, and also of row / A when pairs are rows r and r + 2), (c) the per-thread
row formulas of the four exchange accesses, and checks that (c) equals (b) applied to the plain row,
that the swizzle permutes the rows, that pair partners sit in the same warp at the shuffle distance,
and that the exchange, state-tile and staged-table reads are free of bank conflicts.
"""
import pytest


def split(L):
    A = 16 if L >= 128 else 8 if L >= 32 else 4 if L >= 8 else 2
    return A, L // A


def shape(L):
    A, B = split(L)
    pair = A == 2 * B
    tc0 = 32 if 1024 // L > 32 else (8 if 1024 // L < 8 else 1024 // L)
    tc = 16 if (pair and tc0 > 16) else tc0
    return dict(L=L, A=A, B=B, PAIR=pair, TC=tc, NT=A * tc, SWZ=tc < 16, PNEW=pair and tc <= 8)


def thread(s, tid):
    cl, r = tid % s["TC"], tid // s["TC"]
    if s["PAIR"]:
        if s["PNEW"]:
            xr, xh = (r & 1) | ((r >> 2) << 1), (r >> 1) & 1
        else:
            xr, xh = r >> 1, r & 1
    else:
        xr, xh = r, 0
    return cl, r, xr, xh


def flip(s, row):
    if not s["SWZ"]:
        return 0
    f = (row // s["B"]) & 1
    if s["PNEW"]:
        f ^= (row // s["A"]) & 1
    return f


# the kernel's per-thread forms (xo_inv_st, xo_inv_ld, xo_fwd_st, xo_fwd_ld), as swizzled rows
def inv_st(s, r, k):
    A, B = s["A"], s["B"]
    f = ((k if (A // B) % 2 else 0) + r // B + (k if s["PNEW"] else 0)) & 1 if s["SWZ"] else 0
    return k * A + (r ^ f)


def inv_ld(s, r, xr, xh, t):  # PAIR: t = 2q
    A, B = s["A"], s["B"]
    if s["PAIR"]:
        f = ((1 if t // 2 >= B // 2 else 0) ^ ((xr & 1) if s["PNEW"] else 0)) if s["SWZ"] else 0
        return xr * A + t + (xh ^ f)
    f = (((r if (A // B) % 2 else 0) + t // B) & 1) if s["SWZ"] else 0
    return r * A + (t ^ f)


def fwd_st(s, r, xr, xh, k):
    B = s["B"]
    if s["PAIR"]:
        return 2 * k * B + xh * B + (xr ^ ((xh ^ ((k & 1) if s["PNEW"] else 0)) if s["SWZ"] else 0))
    return k * B + (r ^ ((k & 1) if s["SWZ"] else 0))


def fwd_ld(s, r, t):
    B = s["B"]
    return r * B + (t ^ (((r ^ ((r >> 1) if s["PNEW"] else 0)) & 1) if s["SWZ"] else 0))


def accesses(s):
    """(name, width in 4-byte words, [per-thread word address or None]) per access instruction."""
    A, B, TC, NT, L = s["A"], s["B"], s["TC"], s["NT"], s["L"]
    XN = A // 2 if s["PAIR"] else A
    th = [thread(s, t) for t in range(NT)]
    out = []
    for k in range(B):
        out.append(("inv_st", 2, [2 * (inv_st(s, r, k) * TC + cl) for cl, r, xr, xh in th]))
    if s["PAIR"]:
        for q in range(XN):
            out.append(("inv_ld", 2, [2 * (inv_ld(s, r, xr, xh, 2 * q) * TC + cl) for cl, r, xr, xh in th]))
        for k in range(XN):
            out.append(("fwd_st", 2, [2 * (fwd_st(s, r, xr, xh, k) * TC + cl) for cl, r, xr, xh in th]))
    else:
        for t in range(A):
            out.append(("inv_ld", 2, [2 * (inv_ld(s, r, xr, xh, t) * TC + cl) if r < B else None
                                      for cl, r, xr, xh in th]))
        for k in range(A):
            out.append(("fwd_st", 2, [2 * (fwd_st(s, r, xr, xh, k) * TC + cl) if r < B else None
                                      for cl, r, xr, xh in th]))
    for t in range(B):
        out.append(("fwd_ld", 2, [2 * (fwd_ld(s, r, t) * TC + cl) for cl, r, xr, xh in th]))
    xpos = (lambda q, r, xr, xh: xr + B * (XN * xh + q)) if s["PAIR"] else (lambda q, r, xr, xh: r + B * q)
    upper = (lambda q, xh: xh) if s["PAIR"] else (lambda q, xh: 1 if q >= XN // 2 else 0)
    act = (lambda r: True) if s["PAIR"] else (lambda r: r < B)
    for q in range(XN):
        out.append(("state_ld", 2, [2 * (xpos(q, r, xr, xh) * TC + cl) if act(r) else None
                                    for cl, r, xr, xh in th]))
        out.append(("coef_ld", 1, [xpos(q, r, xr, xh) + 2 * upper(q, xh) if act(r) else None
                                   for cl, r, xr, xh in th]))
    return out


def worst_conflict(width, addrs):
    """Largest number of distinct words one bank serves in one wavefront (8-byte accesses are
    serviced per half-warp, 4-byte ones per warp)."""
    worst = 1
    for w0 in range(0, len(addrs), 32):
        warp = addrs[w0:w0 + 32]
        groups = [warp[:16], warp[16:]] if width == 2 else [warp]
        for g in groups:
            banks = {}
            for a in g:
                if a is None:
                    continue
                for i in range(width):
                    banks.setdefault((a + i) % 32, set()).add(a + i)
            if banks:
                worst = max(worst, max(len(v) for v in banks.values()))
    return worst


SHAPES = [shape(L) for L in (8, 16, 32, 64, 128, 256)]  # every instantiated line length


@pytest.mark.parametrize("s", SHAPES, ids=[f"L{s['L']}" for s in SHAPES])
def test_per_thread_rows_equal_generic_swizzle(s):
    A, B, NT = s["A"], s["B"], s["NT"]
    XN = A // 2 if s["PAIR"] else A
    for tid in range(NT):
        cl, r, xr, xh = thread(s, tid)
        for k in range(B):
            row = k * A + r
            assert inv_st(s, r, k) == row ^ flip(s, row)
        for t in range(B):
            row = r * B + t
            assert fwd_ld(s, r, t) == row ^ flip(s, row)
        if s["PAIR"]:
            for q in range(XN):
                row = xr * A + 2 * q + xh
                assert inv_ld(s, r, xr, xh, 2 * q) == row ^ flip(s, row)
                row = (2 * q + xh) * B + xr
                assert fwd_st(s, r, xr, xh, q) == row ^ flip(s, row)
        elif r < B:
            for t in range(A):
                row = r * A + t
                assert inv_ld(s, r, xr, xh, t) == row ^ flip(s, row)
                row = t * B + r
                assert fwd_st(s, r, xr, xh, t) == row ^ flip(s, row)


@pytest.mark.parametrize("s", SHAPES, ids=[f"L{s['L']}" for s in SHAPES])
def test_swizzle_permutes_rows_and_pairs_share_a_warp(s):
    L, A, B, TC, NT = s["L"], s["A"], s["B"], s["TC"], s["NT"]
    assert sorted(r ^ flip(s, r) for r in range(L)) == list(range(L))
    if s["PAIR"]:
        pd = 2 if s["PNEW"] else 1
        seen = set()
        for tid in range(NT):
            cl, r, xr, xh = thread(s, tid)
            p = tid ^ (pd * TC)
            assert p // 32 == tid // 32
            cl2, r2, xr2, xh2 = thread(s, p)
            assert (cl2, xr2, xh2) == (cl, xr, 1 - xh)
            seen.add((cl, xr, xh))
        assert len(seen) == TC * B * 2


@pytest.mark.parametrize("s", SHAPES, ids=[f"L{s['L']}" for s in SHAPES])
def test_shared_memory_accesses_are_conflict_free(s):
    for name, width, addrs in accesses(s):
        assert worst_conflict(width, addrs) == 1, name


def test_pair_layout_matters_at_eight_lines():
    """With pairs of rows r and r + 1 at 8 lines per CTA the state-tile reads would conflict 2-way,
    which the r, r + 2 pairing removes."""
    s = dict(shape(128), PNEW=False)
    worst = max(worst_conflict(w, a) for n, w, a in accesses(s) if n == "state_ld")
    assert worst == 2
