"""Host model of the tiling of the single-kernel FP32 Q2 A apply (q2_fused.cu), checked on the
CPU: for ragged meshes in all three axes and several resident-block counts, every mesh node is
written exactly once (inside a tile's node box by the element kernel, or on a tile surface by the
fix-up kernel), every shell index is in range and written once per tile, and the fix-up reads
exactly the shell entries that the element kernel wrote.  The functions restate the kernels'
index arithmetic (tile choice, surface index, surface-node enumeration, tiles through a node).
"""
import pytest

FBY, FSEG = 4, 32

def shell_index(a, b, c, ax, by, cz):
    px, py = ax + 1, by + 1
    if c == 0: return a + px * b
    if c == cz: return px * py + a + px * b
    base = 2 * px * py + (c - 1) * (2 * px + 2 * (by - 1))
    if b == 0: return base + a
    if b == by: return base + px + a
    assert a == 0 or a == ax
    return base + 2 * px + 2 * (b - 1) + (0 if a == 0 else 1)

def tiles(nx, ny, nz, slots=304):
    nseg = -(-nx // FSEG); nyt = -(-ny // FBY)
    best = None
    for zc in range(min(4, nz), nz + 1):
        nzc = -(-nz // zc); t = nseg * nyt * nzc
        cost = -(-t // slots) * zc
        if best is None or cost <= best: best = cost; ZC = zc
    nzc = -(-nz // ZC)
    px, py = 2 * FSEG + 1, 2 * FBY + 1
    ss = 2 * px * py + (2 * ZC - 1) * (2 * px + 2 * (py - 2))
    NX, NY, NZ = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
    nzf, nyf, nxf = nzc + 1, nyt + 1, nseg + 1
    n1 = nzf * NY * NX; n2 = (NZ - nzf) * nyf * NX; n3 = (NZ - nzf) * (NY - nyf) * nxf
    return dict(zc=ZC, nseg=nseg, nyt=nyt, nzc=nzc, ss=ss, n1=n1, n2=n2, n3=n3)

def span(X, P, nt):
    t1 = min(X // P, nt - 1); l1 = X - P * t1
    two = l1 == 0 and t1 > 0
    return [(t1 - 1, P), (t1, l1)] if two else [(t1, l1)]

def off_face(q, P): return P * (q // (P - 1)) + 1 + q % (P - 1)

def check(nx, ny, nz, slots=304):
    T = tiles(nx, ny, nz, slots)
    NX, NY, NZ = 2 * nx + 1, 2 * ny + 1, 2 * nz + 1
    written = {}
    shell_written = set()
    for tz in range(T['nzc']):
        for ty in range(T['nyt']):
            for ts in range(T['nseg']):
                tile = ts + T['nseg'] * (ty + T['nyt'] * tz)
                nxt = min(FSEG, nx - ts * FSEG); nyt = min(FBY, ny - ty * FBY)
                ez0 = tz * T['zc']; nzt = min(T['zc'], nz - ez0)
                ax, by, cz = 2 * nxt, 2 * nyt, 2 * nzt
                X0, Y0, Z0 = 2 * ts * FSEG, 2 * ty * FBY, 2 * ez0
                zls = list(range(0, 2 * nzt)) + [cz]
                for w in range(nyt):
                    for lane in range(nxt):
                        for Zl in zls:
                            for j in range(3):
                                if j == 2 and w != nyt - 1: continue
                                Yl = 2 * w + j
                                for i in range(3):
                                    if i == 2 and lane != nxt - 1: continue
                                    Xl = 2 * lane + i
                                    face = Zl in (0, cz) or Yl in (0, by) or Xl in (0, ax)
                                    if face:
                                        si = shell_index(Xl, Yl, Zl, ax, by, cz)
                                        assert 0 <= si < T['ss'], (si, T['ss'])
                                        key = (tile, si)
                                        assert key not in shell_written, key
                                        shell_written.add(key)
                                    else:
                                        n = (X0 + Xl) + NX * ((Y0 + Yl) + NY * (Z0 + Zl))
                                        assert n not in written, n
                                        written[n] = 'e'
    # fix-up
    PX, PY, PZ = 2 * FSEG, 2 * FBY, 2 * T['zc']
    nyf, nxf = T['nyt'] + 1, T['nseg'] + 1
    used = set()
    for idx in range(T['n1'] + T['n2'] + T['n3']):
        i2 = idx
        if i2 < T['n1']:
            ix = i2 % NX; r = i2 // NX; iy = r % NY; kf = r // NY
            iz = PZ * kf if kf < T['nzc'] else NZ - 1
        else:
            i2 -= T['n1']
            if i2 < T['n2']:
                ix = i2 % NX; r = i2 // NX; m = r % nyf
                iy = PY * m if m < T['nyt'] else NY - 1
                iz = off_face(r // nyf, PZ)
            else:
                i2 -= T['n2']
                p = i2 % nxf; r = i2 // nxf; nyo = NY - nyf
                ix = PX * p if p < T['nseg'] else NX - 1
                iy = off_face(r % nyo, PY); iz = off_face(r // nyo, PZ)
        assert 0 <= ix < NX and 0 <= iy < NY and 0 <= iz < NZ, (ix, iy, iz)
        n = ix + NX * (iy + NY * iz)
        assert n not in written, ('dup', n, written.get(n))
        written[n] = 'f'
        for tz, zl in span(iz, PZ, T['nzc']):
            cz = 2 * min(T['zc'], nz - tz * T['zc'])
            for ty, yl in span(iy, PY, T['nyt']):
                by = 2 * min(FBY, ny - ty * FBY)
                for tx, xl in span(ix, PX, T['nseg']):
                    ax = 2 * min(FSEG, nx - tx * FSEG)
                    assert 0 <= xl <= ax and 0 <= yl <= by and 0 <= zl <= cz
                    tile = tx + T['nseg'] * (ty + T['nyt'] * tz)
                    key = (tile, shell_index(xl, yl, zl, ax, by, cz))
                    assert key in shell_written, key
                    used.add(key)
    assert len(written) == NX * NY * NZ, (len(written), NX * NY * NZ)
    assert used == shell_written, len(shell_written - used)
    return T


@pytest.mark.parametrize("dims", [(32, 32, 32), (33, 5, 7), (40, 9, 3), (64, 6, 10), (35, 1, 1), (32, 4, 1),
                                  (70, 13, 11), (96, 8, 17), (48, 32, 40)])
@pytest.mark.parametrize("slots", [304, 7, 1])
def test_fused_tiling_covers_every_node_once(dims, slots):
    check(*dims, slots=slots)


def test_fused_tile_chunks():
    # 64^3 on 304 resident blocks: 2 x 16 tiles per chunk, 8 layers a chunk fills one wave
    assert tiles(64, 64, 64)["zc"] == 8
    # 128^3: 4 x 32 tiles per chunk; 5 layers (26 chunks, 3328 tiles, 11 waves: 55 steps per thread)
    assert tiles(128, 128, 128)["zc"] == 5
