"""CPU model of the copy plan of the 3-D strip kernel (step3_strip_kernel,
variants 5 and 6 of lbm3_set_kernel), checked before any GPU run.

The kernel stages every value it reads through 1-D bulk copies of row
segments (cp.async.bulk).  This test restates, in Python, how the kernel
builds each thread's segment descriptor (row and plane of the pull, the
16-byte chunks a population reads, the split at the periodic edge) and how
it issues a stage, then checks on many boxes and tiles that
  * every piece starts and ends on a 16-byte boundary, in global and shared
    memory, and lies inside its array and inside its stage region;
  * the bytes of a stage add up to the count that arms its mbarrier;
  * every shared-memory element a thread reads (the 19 pulled f, phi*u, and
    the 7 g and low part of g_0 of its node and of its halo positions)
    holds the value of the right periodic source node: f_i at x - c_i, and
    so on (pull of Eqs. 20 and 30 on D3Q19 / D3Q7).
No GPU is needed; a mistake here would be an out-of-bounds copy or a wrong
neighbour on the GPU.
"""
import pytest

CX = [0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0]
CY = [0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1]
CZ = [0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1]


def shape(BX, BY, sS, sT=4):
    """Stage layout, as StripShape in lbm3_strip.cuh."""
    ES, ET = 16 // sS, 16 // sT
    WS, WT, NR = BX + 2 * ES, BX + 2 * ET, BY + 2
    F_OFF = 0
    GM_OFF = F_OFF + 19 * BY * WS * sS
    J_OFF = GM_OFF + 6 * NR * WS * sS
    G0_OFF = J_OFF + 3 * BY * BX * sT
    STAGE = G0_OFF + 2 * NR * WT * sT
    TX = ((19 * BX + 10 * ES) * BY + (6 * BX + 10 * ES) * NR) * sS + \
        (3 * BX * BY + 2 * (BX + 2 * ET) * NR) * sT
    return dict(ES=ES, ET=ET, WS=WS, WT=WT, NR=NR, F_OFF=F_OFF, GM_OFF=GM_OFF,
                J_OFF=J_OFF, G0_OFF=G0_OFF, STAGE=STAGE, TX=TX, NQ=22 * BY + 8 * NR)


def descriptors(nx, ny, x0, y0, BX, BY, sS, sT, P):
    """Per-thread segment descriptors of one CTA, as the kernel builds them:
    (array, piece A offset in bytes without the plane offset, stage offset,
    bytes, plane index 0..3 = z-1..z+2, element size, piece B delta, stage
    offset, bytes)."""
    sh = shape(BX, BY, sS, sT)
    ES, ET, WS, WT, NR = sh["ES"], sh["ET"], sh["WS"], sh["WT"], sh["NR"]
    wy = lambda v: v % ny
    out = []
    for q in range(sh["NQ"]):
        if q < 19 * BY:  # f_i of tile row r: row y0 + r - c_iy, plane z - c_iz
            i, r = divmod(q, BY)
            lp, rp = (ES if CX[i] == 1 else 0), (ES if CX[i] == -1 else 0)
            arr, pl, rsel, dz, esz = "f", i, r - CY[i], 1 - CZ[i], sS
            xa, ln = x0 - lp, BX + lp + rp
            dst = sh["F_OFF"] + ((i * BY + r) * WS + (ES - lp)) * sS
        elif q < 19 * BY + 6 * NR:  # mover m of phase-A row r: plane z + 1 - c_mz
            u = q - 19 * BY
            m, r = u // NR + 1, u % NR
            lp, rp = (0 if CX[m] == -1 else ES), (0 if CX[m] == 1 else ES)
            arr, pl, rsel, dz, esz = "g", m - 1, r - 1 - CY[m], 2 - CZ[m], sS
            xa, ln = x0 - lp, BX + lp + rp
            dst = sh["GM_OFF"] + (((m - 1) * NR + r) * WS + (ES - lp)) * sS
        elif q < 22 * BY + 6 * NR:  # phi*u: row y0 + r, plane z
            c, r = divmod(q - 19 * BY - 6 * NR, BY)
            arr, pl, rsel, dz, esz, xa, ln = "J", c, r, 1, sT, x0, BX
            dst = sh["J_OFF"] + (c * BY + r) * BX * sT
        else:  # g_0 (h = 0) and its low part: row y0 - 1 + r, plane z + 1
            h, r = divmod(q - 22 * BY - 6 * NR, NR)
            arr, pl, rsel, dz, esz = ("g0" if h == 0 else "lo"), 0, r - 1, 2, sT
            xa, ln = x0 - ET, BX + 2 * ET
            dst = sh["G0_OFF"] + (h * NR + r) * WT * sT
        row = (pl * P + wy(y0 + rsel) * nx) * esz
        xA, nA, xB, nB, dB = xa, ln, 0, 0, 0
        if xa < 0:  # the left chunk comes from the end of the row
            xB, nB, dB = nx + xa, -xa, dst
            dst += nB * esz
            xA, nA = 0, ln - nB
        elif xa + ln > nx:  # the right chunk comes from the start of the row
            nA = nx - xa
            nB, xB, dB = ln - nA, 0, dst + nA * esz
        assert 0 <= xA and xA + nA <= nx and 0 <= xB and xB + nB <= nx
        out.append((arr, row + xA * esz, dst, nA * esz, dz, esz, (xB - xA) * esz, dB, nB * esz))
    return out


def check_box(nx, ny, nz, BX, BY, sS, sT=4):
    sh = shape(BX, BY, sS, sT)
    assert sh["NQ"] <= BX * BY  # one segment per thread
    for off in ("GM_OFF", "J_OFF", "G0_OFF", "STAGE"):
        assert sh[off] % 16 == 0
    n = nx * ny * nz
    P = (n + 63) // 64 * 64
    planes = {"f": (sS, 19), "g": (sS, 6), "J": (sT, 3), "g0": (sT, 1), "lo": (sT, 1)}
    node = lambda x, y, z: ((z % nz) * ny + (y % ny)) * nx + (x % nx)
    ES, ET, WS, WT, NR = sh["ES"], sh["ET"], sh["WS"], sh["WT"], sh["NR"]
    for x0 in range(0, nx, BX):
        for y0 in range(0, ny, BY):
            desc = descriptors(nx, ny, x0, y0, BX, BY, sS, sT, P)
            for z in range(0, nz, max(1, nz // 4)):
                zq = (z - 1) % nz
                zs = [zq, (zq + 1) % nz, (zq + 2) % nz, (zq + 3) % nz]
                smem, total = {}, 0
                for arr, srcA, dst, nbA, dz, esz, dlt, dB, nbB in desc:
                    src = srcA + zs[dz] * nx * ny * esz
                    for s_, d_, nb in ((src, dst, nbA), (src + dlt, dB, nbB)):
                        if nb == 0:
                            continue
                        assert s_ % 16 == 0 and d_ % 16 == 0 and nb % 16 == 0
                        assert 0 <= d_ and d_ + nb <= sh["STAGE"]
                        es, npl = planes[arr]
                        assert 0 <= s_ and s_ + nb <= npl * P * es
                        for e in range(0, nb, esz):
                            el = (s_ + e) // esz
                            smem[d_ + e] = (arr, el // P, el % P)
                        total += nb
                assert total == sh["TX"]
                for ty in range(BY):  # the nodes a CTA updates read f and phi*u
                    if y0 + ty >= ny:
                        continue
                    for tx in range(BX):
                        X, Y = x0 + tx, y0 + ty
                        for i in range(19):
                            o = sh["F_OFF"] + (i * BY + ty) * WS * sS + (tx - CX[i] + ES) * sS
                            assert smem[o] == ("f", i, node(X - CX[i], Y - CY[i], z - CZ[i]))
                        for c in range(3):
                            o = sh["J_OFF"] + (c * BY + ty) * BX * sT + tx * sT
                            assert smem[o] == ("J", c, node(X, Y, z))
                pos = [(tx, ty) for ty in range(BY) for tx in range(BX)]
                pos += [(h, -1) for h in range(-1, BX + 1)] + [(h, BY) for h in range(-1, BX + 1)]
                pos += [(-1, h) for h in range(BY)] + [(BX, h) for h in range(BY)]
                for xl, yl in pos:  # phase A: own and halo positions of plane z + 1
                    r, X, Y = yl + 1, x0 + xl, y0 + yl
                    o = sh["G0_OFF"] + r * WT * sT + (xl + ET) * sT
                    assert smem[o] == ("g0", 0, node(X, Y, z + 1))
                    o = sh["G0_OFF"] + (NR + r) * WT * sT + (xl + ET) * sT
                    assert smem[o] == ("lo", 0, node(X, Y, z + 1))
                    for m in range(1, 7):
                        o = sh["GM_OFF"] + ((m - 1) * NR + r) * WS * sS + (xl - CX[m] + ES) * sS
                        assert smem[o] == ("g", m - 1, node(X - CX[m], Y - CY[m], z + 1 - CZ[m]))


@pytest.mark.parametrize("box,tile", [((64, 21, 20), (32, 8)), ((128, 10, 13), (64, 4)),
                                      ((192, 17, 9), (64, 4)), ((64, 3, 5), (32, 8)),
                                      ((128, 9, 7), (64, 2)), ((64, 1, 1), (32, 8)),
                                      ((256, 16, 8), (64, 4))])
@pytest.mark.parametrize("sbytes", [2, 4], ids=["f16", "f32"])
def test_strip_copy_plan(box, tile, sbytes):
    check_box(*box, *tile, sbytes)
