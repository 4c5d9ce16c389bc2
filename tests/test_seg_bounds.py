"""Index bounds of the segmented coarse-solve kernels, emulated on the CPU.

The index arithmetic of the complex64 segmented solve (k_seg_chain's producer bulk copies,
consumer reads and writes, shared-memory ring and receive buffers; the grouped fix-up
products of k_seg_fixup (slab bulk copies) and the host's group lists; k_seg_middle; k_seg_products) is restated here from the kernels and every access is checked against its
allocation:
  coupling matrices Lm, Up and the segment products Pf, Pb: nb x B x ldb complex64;
  coarse vectors (p, y, x): nb x ldb;
  a CTA's ring: S slots of R x CW entries; its receive buffers: 2 x ldb entries.
Layouts: the 2D P1 and P2 and 3D P1 coarse grids whose blocks fit the segmented solve, the
cluster sizes the plan tries (phase A: 9, 8, 16 CTAs; phase B: 16 where it fits) and every
plausible number of phase-A clusters per path (the plan takes it from the device's occupancy).
Bulk copies must start on 16-byte boundaries and move multiples of 16 bytes; clusters of one
launch must write disjoint blocks (the two backward paths both copy the middle block, with
the same value).
"""
import pytest

ELEM = 8                              # complex64
SMEM_BUDGET = 227 * 1024 - 1024      # opt-in shared memory per CTA minus the plan's reserve
SOLVE_MAX_WARPS, SEG_WIDE_WARPS, RPW_MAX, SEG_MAX_LDB = 18, 32, 4, 1040


def coarse_layout(dim, order, n):
    """Blocks of `order` lattice lines (2D) or planes (3D) of the coarse lattice."""
    W = order * (n // 2) + 1
    plane = W ** (dim - 1)
    nb = (W + order - 1) // order
    B = order * plane
    ldb = (B + 1) & ~1
    return nb, B, ldb


def solve_geometry(B, ldb, CS, CW, S, nrx):
    al = lambda x: (x + 127) & ~127  # noqa: E731
    R = (B + CS - 1) // CS
    o = al(16 * S)                  # full[S], empty[S]
    o = al(o + 32)                  # error word, units issued
    o = al(o + 8 * nrx)             # receive barriers, one per gathering step
    o_gath = o
    o = al(o + ELEM * 2 * ldb)      # receive buffers
    o = al(o)                       # no forward-value rows
    o_stage = o
    o = al(o + ELEM * S * R * CW)
    return dict(R=R, CW=CW, nchunk=(ldb + CW - 1) // CW, S=S, off_gath=o_gath, off_stage=o_stage, total=o)


def seg_geom(B, ldb, CS, nb):
    """Chunk width and ring depth the plan picks for a cluster of CS CTAs (None: none fits)."""
    R = (B + CS - 1) // CS
    wide = SOLVE_MAX_WARPS <= R < SEG_WIDE_WARPS
    nwc = R if wide else min(SOLVE_MAX_WARPS - 1, max(4, R))
    if (R + nwc - 1) // nwc > RPW_MAX:
        return None
    rpw = 1 if wide or (R + nwc - 1) // nwc == 1 else RPW_MAX
    cw = ldb
    while cw >= 2:
        for S in (4, 3, 2):
            G = solve_geometry(B, ldb, CS, cw, S, nb // 2 + 2)
            if G["total"] <= SMEM_BUDGET:
                G.update(CS=CS, nwc=nwc, rpw=rpw, threads=32 * (nwc + 1), nrx=nb // 2 + 2)
                return G
        if cw == 2:
            break
        cw = ((cw // 2) + 1) & ~1
    return None


def make_path(J0, step, n, kmax, kc0):
    k0 = max(1, min(kmax, n))
    ls = (n + k0 - 1) // k0
    return dict(J0=J0, step=step, n=n, Ls=ls, K=(n + ls - 1) // ls, kc0=kc0)


def seg_end(k, ls, n):
    return min((k + 1) * ls, n) - 1


def blk(p, q):
    return p["J0"] + p["step"] * q


def seg_paths(nb, K):
    m = nb // 2
    f0 = make_path(0, 1, m, K, 0)
    f1 = make_path(nb - 1, -1, nb - 1 - m, K, f0["K"])
    b0 = make_path(m, -1, m + 1, K, 0)
    b1 = make_path(m, 1, nb - m, K, b0["K"])
    return m, (f0, f1), (b0, b1)


def check_chain(nb, B, ldb, G, pp, phase):
    """One launch of k_seg_chain; returns {cluster: set of blocks it writes}."""
    CS, R, CW, S, nchunk = G["CS"], G["R"], G["CW"], G["S"], G["nchunk"]
    nwc, rpw = G["nwc"], G["rpw"]
    assert G["threads"] <= 1024 and G["total"] <= SMEM_BUDGET
    assert G["off_gath"] % 16 == 0 and G["off_stage"] % 16 == 0
    mat_size, vec_size = nb * B * ldb, nb * ldb
    nr_of = [max(0, min(B, r * R + R) - r * R) for r in range(CS)]
    assert sum(nr_of) == B                             # each CTA receives B values per step
    nclusters = pp[0]["K"] + pp[1]["K"] if phase == 0 else 2
    writes = {}
    for cid in range(nclusters):
        pi = (1 if cid >= pp[1]["kc0"] else 0) if phase == 0 else cid
        p = pp[pi]
        seg = cid - p["kc0"] if phase == 0 else 0
        assert 0 <= seg < p["K"]
        q0 = seg * p["Ls"]
        nsteps = max(0, min(p["Ls"], p["n"] - q0)) if phase == 0 else p["K"] - 1
        pos = (lambda t: q0 + t) if phase == 0 else (lambda t: seg_end(t + 1, p["Ls"], p["n"]))
        tm = 1 if phase == 0 else 0
        assert nsteps - 1 <= G["nrx"]                  # one receive barrier per gathering step
        writes[cid] = set()
        if phase == 1 and nsteps > 0:
            x0 = blk(p, seg_end(0, p["Ls"], p["n"]))
            assert 0 <= x0 < nb and x0 * ldb + B <= vec_size and ldb + B <= 2 * ldb
        for rank in range(CS):
            r0, nr = rank * R, nr_of[rank]
            for t in range(nsteps):
                J = blk(p, pos(t))
                assert 0 <= J < nb
                if phase == 1:
                    assert pos(t) == seg_end(t + 1, p["Ls"], p["n"])
                for r in (0, nr - 1, rpw * nwc - 1):   # right-hand-side prefetch (clamped rows)
                    assert 0 <= J * ldb + (r0 + r if 0 <= r < nr else 0) < vec_size
                if nr:
                    assert r0 + nr <= B and J * ldb + r0 + nr <= vec_size   # output rows
                    assert (t & 1) * ldb + r0 + nr <= 2 * ldb               # receive buffer
                    assert rpw * nwc >= nr                                  # every row owned
                    writes[cid].add(J)
                if t >= tm and nr:
                    base = J * B * ldb + r0 * ldb
                    if nchunk == 1:
                        nbytes = ELEM * nr * ldb
                        assert nbytes % 16 == 0 and (base * ELEM) % 16 == 0
                        assert base + nr * ldb <= mat_size and nr * ldb <= R * CW
                        assert nbytes < (1 << 20)                        # transaction count
                    else:
                        for c in range(nchunk):
                            c0 = c * CW
                            nc = min(CW, ldb - c0)
                            assert nc > 0 and (nc * ELEM) % 16 == 0
                            assert ((base + c0) * ELEM) % 16 == 0 and (CW * ELEM) % 16 == 0
                            assert base + (nr - 1) * ldb + c0 + nc <= mat_size
                            assert (nr - 1) * CW + nc <= R * CW
    return writes


def check_disjoint(writes, allowed):
    seen = {}
    for cid, blocks in writes.items():
        for J in blocks:
            if J in seen:
                assert J in allowed, f"block {J} written by clusters {seen[J]} and {cid}"
            seen[J] = cid


GROUP = 4                             # vectors per group of the grouped block products
GROUP_SMEM = 48 * 1024


def group_cap(ldb, elem):
    row = elem * ldb
    return 4 if 4 * row <= GROUP_SMEM else 2 if 2 * row <= GROUP_SMEM else 1 if row <= GROUP_SMEM else 0


def pack_groups(items, cap):
    """(matrix block, source, destination) items packed as groups of at most cap items sharing a
    matrix block, in the order of each block's first use; unused slots repeat the last item."""
    uses = {}
    for it in items:
        uses.setdefault(it[0], []).append(it)
    groups = []
    for mb, lst in uses.items():
        for b in range(0, len(lst), cap):
            chunk = lst[b:b + cap]
            pad = chunk + [chunk[-1]] * (GROUP - len(chunk))
            groups.append((mb, len(chunk), [it[1] for it in pad], [it[2] for it in pad]))
    return groups


SLAB_CHUNKS, SLAB_MAX_ROWS, SLAB_BYTES = 4, 32, 64 * 1024


def slab_rows(B, ldb, elem):
    """Rows per CTA of the grouped products (the host's grows)."""
    smax = max(1, min(SLAB_MAX_ROWS, SLAB_BYTES // (ldb * elem)))
    nslab = -(-B // smax)
    return -(-B // nslab)


def group_smem(cap, ldb, elem, rows):
    return 128 + ((elem * cap * ldb + 127) & ~127) + elem * rows * ldb


def check_group_launch(groups, nb, B, ldb, cap, elem, sub):
    """k_block_gemv / k_seg_fixup over a group list: the vectors' and the slab's bulk copies,
    matrix rows, outputs."""
    mat_size, vec_size = nb * B * ldb, nb * ldb
    assert cap in (1, 2, 4) and cap * ldb * elem <= GROUP_SMEM and ldb % 2 == 0
    rows = slab_rows(B, ldb, elem)
    assert group_smem(cap, ldb, elem, rows) <= SMEM_BUDGET
    slabs = [(a0, min(B, a0 + rows)) for a0 in range(0, B, rows)]
    assert all(a1 > a0 for a0, a1 in slabs)                # no empty slab (every CTA has rows)
    srcs, dsts = set(), set()
    for mb, g, src, dst in groups:
        assert 1 <= g <= cap and 0 <= mb < nb
        gpad = 4 if g == 3 else g                     # three vectors run as four (a zero fourth)
        assert gpad <= cap                            # shared memory holds gpad staged vectors
        G = 1 if g == 1 else 2 if g == 2 else 4       # the group_rows instance
        assert g <= G <= cap
        for v in range(g):
            assert 0 <= src[v] < nb and 0 <= dst[v] < nb
            assert src[v] * ldb + B <= vec_size and dst[v] * ldb + B <= vec_size
            # the vector's bulk copy: ldb entries from src[v] ldb into staged slot v
            assert src[v] * ldb + ldb <= vec_size and (src[v] * ldb * elem) % 16 == 0 and (ldb * elem) % 16 == 0
            assert dst[v] not in dsts                 # each destination written by one CTA column
            dsts.add(dst[v])
            srcs.add(src[v])
        assert g * ldb * elem < (1 << 20)             # the vectors' barrier transaction count
    mbs = [gr[0] for gr in groups]
    for mb in {min(mbs), max(mbs)} if mbs else ():    # copies are affine in mb: check the extremes
        for a0, a1 in slabs:                           # the slab's bulk copies, chunk by chunk
            nr = a1 - a0
            rpc = -(-nr // SLAB_CHUNKS)
            covered = 0
            for c in range(SLAB_CHUNKS):
                r0 = min(nr, c * rpc)
                r1 = min(nr, r0 + rpc)
                nbytes = elem * (r1 - r0) * ldb
                src = ((mb * B + a0) + r0) * ldb
                assert nbytes % 16 == 0 and (src * elem) % 16 == 0 and nbytes < (1 << 20)
                assert src + (r1 - r0) * ldb <= mat_size and r1 * ldb <= rows * ldb
                covered += r1 - r0
            assert covered == nr
    if sub:
        assert not srcs & dsts                        # sources are read while destinations change
    return dsts


def check_fixup_middle_products(nb, B, ldb, m, pp, pmap=None):
    mat_size, vec_size = nb * B * ldb, nb * ldb
    assert ldb <= SEG_MAX_LDB
    cap = group_cap(ldb, ELEM)
    items = []
    for p in pp:                                      # the host's group list of the fix-ups
        for q in range(p["Ls"], p["n"]):
            k = q // p["Ls"]
            if q == seg_end(k, p["Ls"], p["n"]):
                continue                              # a segment's end: phase B
            J = blk(p, q)
            items.append((pmap[J] if pmap else J, blk(p, k * p["Ls"] - 1), J))
    fixed = check_group_launch(pack_groups(items, cap), nb, B, ldb, cap, ELEM, True)
    for p in pp:
        for q in range(p["Ls"], p["n"]):              # every non-end position of k >= 1 fixed
            k = q // p["Ls"]
            if q != seg_end(k, p["Ls"], p["n"]):
                assert blk(p, q) in fixed
    for p in pp:                                      # k_seg_products, one z-slice per segment
        for k in range(1, p["K"]):
            for i in range(p["Ls"]):
                q = k * p["Ls"] + i
                if q > seg_end(k, p["Ls"], p["n"]):
                    continue
                J = blk(p, q)
                assert 0 <= J < nb and (J + 1) * B * ldb <= mat_size and J != m
                if i:
                    assert 0 <= blk(p, q - 1) < nb
    assert 1 <= m <= nb - 2                           # k_seg_middle reads blocks m-1, m+1
    assert ((m + 1) * B) * ldb <= mat_size and (m + 2) * ldb <= vec_size


LAYOUTS = [(2, 1, n) for n in (30, 32, 36, 48, 64, 100, 128, 256, 512, 1024, 2046)] + \
          [(2, 2, n) for n in (32, 44, 64, 128, 256, 512)] + \
          [(3, 1, n) for n in (30, 32, 40, 48, 60, 62)] + \
          [(2, 3, n) for n in (32, 34, 64, 128)]   # Q3: blocks of three lattice lines


@pytest.mark.parametrize("dim,order,n", LAYOUTS, ids=lambda v: str(v))
def test_segment_kernels_stay_in_bounds(dim, order, n):
    nb, B, ldb = coarse_layout(dim, order, n)
    if nb < 16 or ldb > SEG_MAX_LDB:
        pytest.skip("the plan does not take the segmented solve for this layout")
    checked = 0
    for CS in (9, 8, 16):
        GA = seg_geom(B, ldb, CS, nb)
        if GA is None:
            continue
        GBs = [GA] + ([seg_geom(B, ldb, 16, nb)] if CS != 16 and seg_geom(B, ldb, 16, nb) else [])
        for K in (2, 3, 4, 5, 6, 7, 8, 9, 11, 13, 16, 19, 24, 32, 40):
            m, f, b = seg_paths(nb, K)
            for pp, allowed in ((f, set()), (b, {m})):
                check_disjoint(check_chain(nb, B, ldb, GA, pp, 0), allowed)
                for GB in GBs:
                    check_disjoint(check_chain(nb, B, ldb, GB, pp, 1), set())
                check_fixup_middle_products(nb, B, ldb, m, pp)
                for ctop, cbot in converged_points(nb, m):
                    cmap = block_map(nb, m, ctop, cbot)
                    check_fixup_middle_products(nb, B, ldb, m, pp, product_map(nb, pp, cmap))
            checked += 1
    assert checked > 0


def converged_points(nb, m):
    """Blocks at which the top and bottom chains' Schur inverses are taken as converged."""
    return [(c, nb - 1 - c) for c in (1, 2, 5, m // 2) if 1 <= c < m and m < nb - 1 - c <= nb - 2]


def block_map(nb, m, ctop, cbot):
    """Host cmap: later blocks of a converged chain use the converged block."""
    cmap = list(range(nb))
    for J in range(ctop + 1, m):
        cmap[J] = ctop
    for J in range(m + 1, cbot):
        cmap[J] = cbot
    return cmap


def product_map(nb, pp, cmap):
    """Host pmap of one sweep: the run of segments k >= 1 whose blocks all repeat a converged
    block; its first segment is computed and the rest repeat it position by position."""
    pm = list(range(nb))
    for p in pp:
        kstar, lo, hi = -1, 1, 0
        for k in range(1, p["K"]):
            rep = all(cmap[blk(p, q)] != blk(p, q) for q in range(k * p["Ls"], seg_end(k, p["Ls"], p["n"]) + 1))
            if rep and kstar < 0:
                kstar = k
            elif rep:
                lo = k if lo > hi else lo
                hi = k
            elif kstar >= 0:
                break
        for k in range(lo, hi + 1):
            for q in range(k * p["Ls"], seg_end(k, p["Ls"], p["n"]) + 1):
                pm[blk(p, q)] = blk(p, kstar * p["Ls"] + (q - k * p["Ls"]))
    return pm


GEMV_LAYOUTS = [(2, 1, n) for n in (8, 30, 64, 512, 1024, 2046)] + [(2, 2, n) for n in (8, 64, 512, 1024)] + \
               [(3, 1, n) for n in (8, 32, 62, 96)] + [(2, 3, n) for n in (16, 128)]


@pytest.mark.parametrize("dim,order,n", GEMV_LAYOUTS, ids=lambda v: str(v))
@pytest.mark.parametrize("elem", [8, 16], ids=["complex64", "complex128"])
def test_grouped_prepass_stays_in_bounds(dim, order, n, elem):
    """k_block_gemv's groups p_J = Dinv[cmap J] r_J cover every block once, with and without
    converged chains (blocks wider than 48 KB of shared memory take the wide kernel instead)."""
    nb, B, ldb = coarse_layout(dim, order, n)
    cap = group_cap(ldb, elem)
    if cap == 0:
        assert elem * ldb > GROUP_SMEM
        return
    m = nb // 2 if nb >= 4 else nb - 1
    maps = [list(range(nb))] + [block_map(nb, m, c, b) for c, b in converged_points(nb, m)]
    for cmap in maps:
        groups = pack_groups([(cmap[J], J, J) for J in range(nb)], cap)
        assert check_group_launch(groups, nb, B, ldb, cap, elem, False) == set(range(nb))
        assert len(groups) <= nb and all(g[2] == g[3] for g in groups)


def test_pack_groups_shares_repeated_blocks():
    items = [(7, J, J) for J in range(10)] + [(3, 10, 10)]
    groups = pack_groups(items, 4)
    assert [(g[0], g[1]) for g in groups] == [(7, 4), (7, 4), (7, 2), (3, 1)]
    assert groups[2][2] == [8, 9, 9, 9] and groups[3][3] == [10, 10, 10, 10]
