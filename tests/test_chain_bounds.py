"""Index bounds of the non-segmented coarse-solve kernels, emulated on the CPU.

k_coarse_solve (used by the FP64 form everywhere and by the complex64 form where segments do
not apply: the single chain in one launch, mode 0, or the twisted form as three launches, the
forward chains of both clusters, mode 1, the middle block, and the backward chains, mode 2) and
k_coarse_solve_grid (the whole-grid chain for blocks too large for one cluster) are restated
here from the kernels, and every access is checked against its allocation:
  coupling matrices Lm, Up: nb x B x ldb values; coarse vectors uc: nb x ldb; a CTA's ring:
  S slots of R x CW; its receive buffers 2 x ldb; the forward values wrows (single chain
  only): nb x R; the grid kernel's staged vector: ldb.
Bulk copies must start on 16-byte boundaries and move multiples of 16 bytes. Within one launch
each block is written by at most one cluster, every block's solution is written exactly once
by the backward launch (or the single chain) and the middle kernel, and the blocks visited
follow the forward / middle / backward order of the twisted elimination.
Layouts: 2D P1 and P2, 3D P1, from small meshes up to the serving trace's largest (n = 1024),
for complex64 and complex128, every cluster size the planner tries, one and two chains.
All index expressions are affine in the block index with non-negative coefficients, so the
per-rank checks are made at the first and last block a chain visits.
"""
import pytest

SMEM_BUDGET = 227 * 1024 - 1024      # opt-in shared memory per CTA minus the planner's reserve
SOLVE_MAX_WARPS, RPW_MAX = 18, 4


def coarse_layout(dim, order, n):
    """Blocks of `order` lattice lines (2D) or planes (3D) of the coarse lattice."""
    W = order * (n // 2) + 1
    plane = W ** (dim - 1)
    nb = (W + order - 1) // order
    B = order * plane
    ldb = (B + 1) & ~1
    return nb, B, ldb


def chain_rx(nb, single):
    """Receive barriers of a chain launch (one per gathering step, an upper bound)."""
    return 2 * nb if single else nb // 2 + 2


def solve_geometry(B, ldb, nb, CS, CW, S, elem, with_w):
    al = lambda x: (x + 127) & ~127  # noqa: E731
    R = (B + CS - 1) // CS
    o = al(16 * S)
    o = al(o + 32)
    o = al(o + 8 * chain_rx(nb, with_w))     # receive barriers
    off_gath = o
    o = al(o + elem * 2 * ldb)
    off_w = o
    o = al(o + (elem * nb * R if with_w else 0))
    off_stage = o
    o = al(o + elem * S * R * CW)
    return dict(R=R, CW=CW, S=S, nchunk=(ldb + CW - 1) // CW, off_gath=off_gath, off_w=off_w,
                off_stage=off_stage, total=o)


def cluster_geometries(B, ldb, nb, elem):
    """Every (CS, geometry) the planner's cluster loop can pick (it takes the first one the
    device's occupancy accepts, which the CPU cannot know, so all that fit are checked). The
    single chain (nb < 4) keeps its forward values in shared memory; the twisted form does not."""
    with_w = nb < 4
    out = []
    for CS in (16, 8, 4, 2, 1):
        R = (B + CS - 1) // CS
        nwc = min(SOLVE_MAX_WARPS - 1, max(4, R))
        if (R + nwc - 1) // nwc > RPW_MAX:
            continue
        cw = ldb
        while cw >= 2:
            G = next((solve_geometry(B, ldb, nb, CS, cw, S, elem, with_w) for S in (4, 3, 2)
                      if solve_geometry(B, ldb, nb, CS, cw, S, elem, with_w)["total"] <= SMEM_BUDGET), None)
            if G is not None:
                rpw = 1 if (R + nwc - 1) // nwc == 1 else RPW_MAX
                G.update(CS=CS, nwc=nwc, rpw=rpw, threads=32 * (nwc + 1))
                out.append(G)
                break
            if cw == 2:
                break
            cw = ((cw // 2) + 1) & ~1
    return out


def chain_blocks(nb, mid, cid):
    """Blocks visited by chain cid at steps t = 0 .. 2 nf (forward, middle, backward)."""
    direction, J0 = (1, 0) if cid == 0 else (-1, nb - 1)
    nf = mid if cid == 0 else nb - 1 - mid
    return nf, [J0 + direction * t if t < nf else (mid if t == nf else mid - direction * (t - nf))
                for t in range(2 * nf + 1)]


def chain_steps(nb, mid, cid, mode):
    """Global steps t of one launch of chain cid: mode 0 all of them (single chain), mode 1 the
    forward steps t < nf, mode 2 the backward steps t > nf."""
    nf, blocks = chain_blocks(nb, mid, cid)
    tbeg = nf + 1 if mode == 2 else 0
    tend = nf if mode == 1 else 2 * nf + 1
    return nf, blocks, list(range(tbeg, tend))


def check_cluster_chain(nb, B, ldb, elem, G, ncl):
    """The launches of k_coarse_solve for ncl chains (1: mode 0, single top-down chain,
    mid = nb - 1; 2: twisted, mid = nb / 2, modes 1 and 2 around the middle kernel)."""
    CS, R, CW, S, nchunk, nwc, rpw = (G[k] for k in ("CS", "R", "CW", "S", "nchunk", "nwc", "rpw"))
    assert G["threads"] <= 1024 and G["total"] <= SMEM_BUDGET
    assert G["off_gath"] % 16 == 0 and G["off_w"] % 16 == 0 and G["off_stage"] % 16 == 0
    assert (G["off_w"] == G["off_stage"]) == (ncl == 2)     # forward rows only for the single chain
    mat, vec = nb * B * ldb, nb * ldb
    mid = nb // 2 if ncl == 2 else nb - 1
    nr_of = [max(0, min(B, r * R + R) - r * R) for r in range(CS)]
    assert sum(nr_of) == B                                # each CTA receives B values per step
    final = {}                                            # block -> launch that writes its solution
    for mode in ((0,) if ncl == 1 else (1, 2)):
        writers = {}
        for cid in range(ncl):
            nf, blocks, steps = chain_steps(nb, mid, cid, mode)
            assert all(0 <= J < nb for J in blocks)
            assert len(steps) - 1 <= chain_rx(nb, ncl == 1)    # one receive barrier per gathering step
            fwd, bwd = blocks[:nf], blocks[nf + 1:]
            assert bwd == fwd[::-1] and blocks[nf] == mid      # backward retraces the forward blocks
            if mode == 0:
                written = bwd + [mid]                           # forward values go to wrows
                assert nf <= nb                                 # wrows rows t < nf, read at 2nf - t
            else:
                written = [blocks[t] for t in steps]
                assert mid not in written                       # the middle kernel's block
            for J in written:
                assert J not in writers, (mode, J, writers.get(J), cid)
                writers[J] = cid
                if mode != 1:
                    final[J] = mode
            if mode == 2 and steps:
                assert mid * ldb + B <= vec                     # x_m staged from uc
            visited = [blocks[t] for t in steps] + ([blocks[steps[-1] + 1]] if steps and
                                                    steps[-1] + 1 < len(blocks) else [])
            if not visited:
                continue
            for rank in range(CS):
                r0, nr = rank * R, nr_of[rank]
                assert rpw * nwc >= nr                          # every row of the slice has an owner
                for J in (min(visited), max(visited)):
                    for r in (0, nr - 1, rpw * nwc - 1):        # prefetch: rows outside read entry 0
                        assert 0 <= J * ldb + (r0 + r if 0 <= r < nr else 0) < vec
                    if not nr:
                        continue
                    assert J * ldb + r0 + nr <= vec and r0 + nr <= B <= ldb
                    assert mode != 0 or nf == 0 or (nf - 1) * R + nr <= nb * R   # wrows
                    base = (J * B + r0) * ldb                              # producer's source rows
                    if nchunk == 1:
                        nbytes = elem * nr * ldb
                        assert (base * elem) % 16 == 0 and nbytes % 16 == 0 and nbytes < (1 << 20)
                        assert base + nr * ldb <= mat and nr * ldb <= R * CW
                    else:
                        for c in range(nchunk):
                            c0 = c * CW
                            nc = min(CW, ldb - c0)
                            assert nc > 0 and (nc * elem) % 16 == 0 and ((base + c0) * elem) % 16 == 0
                            assert base + (nr - 1) * ldb + c0 + nc <= mat and (nr - 1) * CW + nc <= R * CW
    if ncl == 2:
        final[mid] = "middle"
    assert sorted(final) == list(range(nb))                 # every block solved exactly once


def check_grid_chain(nb, B, ldb, elem):
    """k_coarse_solve_grid: one chain, mid = nb - 1, vector staged in ldb values of shared memory."""
    if elem * ldb > SMEM_BUDGET:
        return False                                        # the planner returns HELM_ENOTSUP
    nf, blocks = chain_blocks(nb, nb - 1, 0)
    assert all(0 <= J < nb for J in blocks) and len(blocks) == 2 * nf + 1
    for t, J in enumerate(blocks):
        if t >= 1:
            prev = blocks[t - 1]
            assert prev * ldb + B <= nb * ldb               # staged x: entries < B from uc
            assert (J * B + B - 1) * ldb + ldb <= nb * B * ldb   # rows a < B of the coupling block
        assert J * ldb + B <= nb * ldb                      # in-place update of uc rows a < B
    return True


LAYOUTS = [(2, 1, n) for n in (8, 10, 16, 30, 36, 64, 128, 256, 512, 1024)] + \
          [(2, 2, n) for n in (8, 12, 22, 64, 128, 256, 512, 1024)] + \
          [(3, 1, n) for n in (8, 12, 16, 32, 48, 96)] + \
          [(2, 3, n) for n in (8, 16, 18, 32, 64, 128)]   # Q3: blocks of three lattice lines


@pytest.mark.parametrize("dim,order,n", LAYOUTS, ids=lambda v: str(v))
@pytest.mark.parametrize("elem", [8, 16], ids=["complex64", "complex128"])
def test_chain_kernels_stay_in_bounds(dim, order, n, elem):
    nb, B, ldb = coarse_layout(dim, order, n)
    geoms = cluster_geometries(B, ldb, nb, elem)
    for G in geoms:
        check_cluster_chain(nb, B, ldb, elem, G, 2 if nb >= 4 else 1)
    if not geoms:
        # blocks too large for a cluster: the whole-grid chain, or HELM_ENOTSUP beyond its limit
        assert check_grid_chain(nb, B, ldb, elem) or elem * ldb > SMEM_BUDGET
    else:
        check_grid_chain(nb, B, ldb, elem)


def test_large_blocks_take_the_grid_chain():
    """The layouts whose blocks no cluster can hold are the ones the grid chain serves."""
    for dim, order, n in ((2, 2, 1024), (3, 1, 96)):
        for elem in (8, 16):
            nb, B, ldb = coarse_layout(dim, order, n)
            assert not cluster_geometries(B, ldb, nb, elem), (dim, order, n, elem)
            assert check_grid_chain(nb, B, ldb, elem)
