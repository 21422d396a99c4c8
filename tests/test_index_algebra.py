"""The address algebra the size-specialised in-place kernel relies on, checked
on the CPU for every size, precision, cluster size and field count.

The kernel (paper_2410_02532_gb300/csrc/opo_fused2.cuh) stores a column (row)
of the four-step transform XOR-swizzled within 2^SW-element groups:
element e of line l of field f sits at

    f NC + l L + (e ^ (((e >> SW) ^ perm(l)) & (2^SW - 1)))

Two rewritings of that formula are used in the hot loops instead of the
formula itself:

* an in-place work item touches the elements e0 | x of one line, x = r R a
  compile-time constant with bits disjoint from e0; element e0 | x is read at
  the byte offset (a0 ^ lo(x)) + hi(x) from the item's first element's byte
  offset a0 (one logic operation per access);
* a cluster push (one- and two-CTA clusters) finds the destination CTA and
  the start of the destination line group for its unrolled position r in a
  per-CTA table, and XORs the item's own part of the destination index with
  the table's swizzle term.

Both hold because the swizzle is linear over the bits of the element and line
indices and every buffer and line starts on a 128-byte boundary.  These tests
re-derive each access both ways and compare them element by element.
"""
import numpy as np
import pytest

SIZES = [(6, 6), (6, 7), (7, 7), (7, 8), (8, 8), (8, 9)]


def col_split(LP):
    """[Ra1, Ra2] exponents of the column transform (P = 256 splits [8, 32])."""
    A2 = 5 if LP == 8 else (LP + 1) // 2
    return LP - A2, A2


def row_split(LQ):
    """[Rb1, Rb2] exponents of the row transform (Q = 512 splits [32, 16])."""
    B2 = 4 if LQ == 9 else (LQ + 1) // 2
    return LQ - B2, B2


def layout(LP, LQ, dbl, C, F):
    S = 16 if dbl else 8            # bytes per complex element
    SW = 3 if dbl else 4            # 128-byte bank row = 2^SW elements
    SWM = (1 << SW) - 1
    A1, A2 = col_split(LP)
    B1, B2 = row_split(LQ)
    N = 1 << (LP + LQ)
    NC = N // C
    logC = C.bit_length() - 1

    def perm(x):
        return (((x & 1) << (SW - 1)) | ((x >> 1) & ((1 << (SW - 1)) - 1))) & SWM

    def cidx(f, n1, b):   # column b (P elements), column-major X
        return f * NC + (b << LP) + (n1 ^ (((n1 >> SW) ^ perm(b)) & SWM))

    def ridx(f, row, e):  # row (Q elements), row-major Y
        return f * NC + (row << LQ) + (e ^ (((e >> SW) ^ perm(row)) & SWM))

    return dict(S=S, SW=SW, SWM=SWM, Ra1=1 << A1, Ra2=1 << A2, Rb1=1 << B1, Rb2=1 << B2,
                NC=NC, Pc=(1 << LP) // C, Qc=(1 << LQ) // C, logPc=LP - logC,
                logQc=LQ - logC, LP=LP, LQ=LQ, perm=perm, cidx=cidx, ridx=ridx,
                Xoff=0, Yoff=S * F * NC)


def configs():
    for LP, LQ in SIZES:
        for dbl in (False, True):
            for C in (1, 2, 4, 8, 16):
                if (1 << LP) < C:
                    continue
                for F in (2, 3):
                    yield LP, LQ, dbl, C, F


@pytest.mark.parametrize("LP,LQ", SIZES)
def test_in_place_accesses_are_one_xor_and_an_offset(LP, LQ):
    checked = 0
    for lp, lq, dbl, C, F in configs():
        if (lp, lq) != (LP, LQ):
            continue
        g = layout(LP, LQ, dbl, C, F)
        S, SW, SWM = g["S"], g["SW"], g["SWM"]
        Ra1, Ra2, Rb1, Rb2 = g["Ra1"], g["Ra2"], g["Rb1"], g["Rb2"]

        def ipx(a0, x):
            lo = ((x ^ (x >> SW)) & SWM) * S
            hi = (x & ~SWM) * S
            return (a0 ^ lo) + hi

        # (buffer offset, index function, lines, item starts e0, offsets x):
        # the block-A column load/store, the column stage, the push's local
        # load (columns), the row stage, block B and the inverse push's local
        # load (rows)
        pats = [
            (g["Xoff"], g["cidx"], g["Qc"], [(j, r * Ra2) for j in range(Ra2) for r in range(Ra1)]),
            (g["Xoff"], g["cidx"], g["Qc"], [(j * Ra1, r) for j in range(Ra2) for r in range(Ra1)]),
            (g["Xoff"], g["cidx"], g["Qc"], [(j, r * Ra1) for j in range(Ra1) for r in range(Ra2)]),
            (g["Xoff"], g["cidx"], g["Qc"], [(j * Ra2, r) for j in range(Ra1) for r in range(Ra2)]),
            (g["Yoff"], g["ridx"], g["Pc"], [(j, r * Rb2) for j in range(Rb2) for r in range(Rb1)]),
            (g["Yoff"], g["ridx"], g["Pc"], [(j * Rb1, r) for j in range(Rb2) for r in range(Rb1)]),
            (g["Yoff"], g["ridx"], g["Pc"], [(j, r * Rb1) for j in range(Rb1) for r in range(Rb2)]),
            (g["Yoff"], g["ridx"], g["Pc"], [(j * Rb2, r) for j in range(Rb1) for r in range(Rb2)]),
        ]
        for boff, fn, lines, pairs in pats:
            e0 = np.array([p[0] for p in pairs], dtype=np.int64)
            x = np.array([p[1] for p in pairs], dtype=np.int64)
            assert not np.any(e0 & x)
            for f in range(F):
                for line in range(lines):
                    if fn is g["cidx"]:
                        a0 = boff + S * fn(f, e0, line)
                        want = boff + S * fn(f, e0 | x, line)
                    else:
                        a0 = boff + S * fn(f, line, e0)
                        want = boff + S * fn(f, line, e0 | x)
                    assert np.array_equal(ipx(a0, x), want), (LP, LQ, dbl, C, F, f, line)
                    checked += len(pairs)
    assert checked > 0


@pytest.mark.parametrize("LP,LQ", SIZES)
def test_push_tables_give_the_owner_and_the_index(LP, LQ):
    checked = 0
    for lp, lq, dbl, C, F in configs():
        if (lp, lq) != (LP, LQ) or C > 2:
            continue
        g = layout(LP, LQ, dbl, C, F)
        S, perm = g["S"], g["perm"]
        Ra1, Ra2, Rb1, Rb2 = g["Ra1"], g["Ra2"], g["Rb1"], g["Rb2"]
        Pc, Qc, logPc, logQc = g["Pc"], g["Qc"], g["logPc"], g["logQc"]
        # forward push: column stage output k1 = j + r Ra1 of column n2 goes
        # to row k1 of the owner of that row
        if Pc >= Ra1:
            r = np.arange(Ra2)
            R = (r * Ra1) & (Pc - 1)
            dest, base, xv = (r * Ra1) >> logPc, g["Yoff"] + S * (R << LQ), S * perm(R)
            for c in range(C):
                for f in range(F):
                    for j in range(Ra1):
                        n2 = (c << logQc) + np.arange(Qc)[:, None]
                        a0 = S * g["ridx"](f, j, n2)
                        k1 = j + r * Ra1
                        want_o = g["Yoff"] + S * g["ridx"](f, k1 & (Pc - 1), n2)
                        assert np.array_equal(dest, k1 >> logPc)
                        assert np.array_equal(base + (a0 ^ xv), want_o)
                        checked += Qc * Ra2
        # inverse push: row stage output n2 = j + r Rb2 of row k1 goes to
        # column n2 of its owner
        if Qc >= Rb2:
            r = np.arange(Rb1)
            B = (r * Rb2) & (Qc - 1)
            dest, base, xv = (r * Rb2) >> logQc, g["Xoff"] + S * (B << g["LP"]), S * perm(B)
            for c in range(C):
                for f in range(F):
                    for j in range(Rb2):
                        k1 = (c << logPc) + np.arange(Pc)[:, None]
                        a0 = S * g["cidx"](f, k1, j)
                        n2 = j + r * Rb2
                        want_o = g["Xoff"] + S * g["cidx"](f, k1, n2 & (Qc - 1))
                        assert np.array_equal(dest, n2 >> logQc)
                        assert np.array_equal(base + (a0 ^ xv), want_o)
                        checked += Pc * Rb1
    assert checked > 0


def test_a_plausible_slip_is_caught():
    """The comparison above is sharp: taking the swizzle term of the line
    number out of the table entry (a dropped XOR) changes some offsets."""
    g = layout(7, 7, False, 2, 3)
    S, perm = g["S"], g["perm"]
    Ra1, Ra2, Pc = g["Ra1"], g["Ra2"], g["Pc"]
    r = np.arange(Ra2)
    R = (r * Ra1) & (Pc - 1)
    base = g["Yoff"] + S * (R << g["LQ"])
    n2 = np.arange(g["Qc"])[:, None]
    a0 = S * g["ridx"](0, 1, n2)
    want = g["Yoff"] + S * g["ridx"](0, (1 + r * Ra1) & (Pc - 1), n2)
    assert np.array_equal(base + (a0 ^ (S * perm(R))), want)
    assert not np.array_equal(base + a0, want)


@pytest.mark.parametrize("LP,LQ,dbl", [(8, 9, False), (8, 8, True)])
@pytest.mark.parametrize("F", [2, 3])
def test_global_exchange_covers_every_element_once(LP, LQ, dbl, F):
    """The form that exchanges through global memory (three FP32 fields at
    2^17, FP64 at 2^16; 16 CTAs): the forward push and the inverse push each
    write every element of their buffer exactly once, the row stage and the
    column stage after the barriers read every element exactly once, and each
    CTA's reads fill its whole in-place buffer (Y, then X) exactly once."""
    C = 16
    g = layout(LP, LQ, dbl, C, F)
    Ra1, Ra2, Rb1, Rb2 = g["Ra1"], g["Ra2"], g["Rb1"], g["Rb2"]
    Pc, Qc, logPc, logQc = g["Pc"], g["Qc"], g["logPc"], g["logQc"]
    P, Q = 1 << LP, 1 << LQ
    N = P * Q
    c = np.arange(C)[:, None, None, None, None]
    f = np.arange(F)[None, :, None, None, None]
    # forward push: column b of CTA c, butterfly j < Ra1, output r < Ra2 ->
    # G1[f][k1 = j + r Ra1][n2 = c Qc + b]
    b = np.arange(Qc)[None, None, :, None, None]
    j = np.arange(Ra1)[None, None, None, :, None]
    r = np.arange(Ra2)[None, None, None, None, :]
    w1 = (f * N + (j + r * Ra1) * Q + (c << logQc) + b).ravel()
    assert np.array_equal(np.sort(w1), np.arange(F * N))
    # row stage: CTA c, row < Pc, butterfly j < Rb2, input r < Rb1 reads
    # G1[f][c Pc + row][j + r Rb2] and writes Y element j Rb1 + r of that row
    row = np.arange(Pc)[None, None, :, None, None]
    j = np.arange(Rb2)[None, None, None, :, None]
    r = np.arange(Rb1)[None, None, None, None, :]
    r1 = (f * N + ((c << logPc) + row) * Q + j + r * Rb2).ravel()
    assert np.array_equal(np.sort(r1), np.arange(F * N))
    ya = np.broadcast_to(g["ridx"](f, row, j * Rb1 + r), (C, F, Pc, Rb2, Rb1))
    for cc in range(C):
        assert np.array_equal(np.sort(ya[cc].ravel()), np.arange(F * g["NC"]))
    # inverse push: CTA c, row < Pc, butterfly j < Rb2, output r < Rb1 ->
    # G2[f][n1 = c Pc + row][n2 = j + r Rb2]
    w2 = (f * N + ((c << logPc) + row) * Q + j + r * Rb2).ravel()
    assert np.array_equal(np.sort(w2), np.arange(F * N))
    # column stage: CTA c, column b < Qc, butterfly j < Ra1, input r < Ra2
    # reads G2[f][j + r Ra1][c Qc + b] and writes X element j Ra2 + r of
    # column b
    b = np.arange(Qc)[None, None, :, None, None]
    j = np.arange(Ra1)[None, None, None, :, None]
    r = np.arange(Ra2)[None, None, None, None, :]
    r2 = (f * N + (j + r * Ra1) * Q + (c << logQc) + b).ravel()
    assert np.array_equal(np.sort(r2), np.arange(F * N))
    xa = np.broadcast_to(g["cidx"](f, j * Ra2 + r, b), (C, F, Qc, Ra1, Ra2))
    for cc in range(C):
        assert np.array_equal(np.sort(xa[cc].ravel()), np.arange(F * g["NC"]))
