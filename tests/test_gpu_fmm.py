"""GPU parity of the C-ABI path against the FP64 oracle: all-pairs direct sums (FP64 and
FP32), octree invariants and interaction-list coverage, and the KIFMM evaluation of the
Kelvin sums of Eq. fmm_summation (single layer, double layer, both, and stress).

The oracle always receives exactly the inputs the GPU receives (points, normals and
densities rounded to FP32 first): for near-coincident points the 1/r^2 double layer is as
sensitive to the input rounding as to the arithmetic.

Tolerances: FP64 direct sum 1e-12 relative L2 (rounding order only).  FP32 direct sum 3e-5:
each output sums ~1800 terms with FP32 rounding (~6e-8 each, growing like sqrt(n)) and
clouds with near-coincident points cancel large terms (up to ~10x).  FMM at p = 6
(152-point surfaces): 1e-4 relative L2, the accuracy set for the multipole order.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_04082_gb300 as K
    return K


def dev(a, dtype=torch.float32):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda:0")


def r32(a):
    """The FP32 rounding of an FP64 array, back in FP64 (what the GPU path receives)."""
    return None if a is None else np.asarray(a, np.float32).astype(np.float64)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


G1, NU1 = 1.0, 0.3
G2, NU2 = 2.3, 0.21


def make_ctx(K, G=G1, nu=NU1, **kw):
    f = K.Kfmm(**kw)
    f.set_material(K.material_K(G, nu), G)
    return f


# ----------------------------------------------------------------- direct sums
@pytest.mark.parametrize("kind", ["disp", "stress"])
@pytest.mark.parametrize("layers", ["sl", "dl", "both"])
def test_direct_fp64_and_fp32(K, kind, layers):
    rng = np.random.default_rng(3)
    ns, nt = 1777, 913  # ragged sizes, not multiples of the 256-thread tile
    src = r32(rng.uniform(-1, 1, (ns, 3)))
    trg = np.vstack([r32(rng.uniform(-1, 1, (nt - 5, 3))), src[:5]])  # includes coincident points
    nrm = rng.normal(size=(ns, 3))
    nrm = r32(nrm / np.linalg.norm(nrm, axis=1, keepdims=True))
    sl = r32(rng.normal(size=(ns, 3))) if layers in ("sl", "both") else None
    dl = r32(rng.normal(size=(ns, 3))) if layers in ("dl", "both") else None
    no = 3 if kind == "disp" else 6
    kk = K.KFMM_DISP if kind == "disp" else K.KFMM_STRESS
    f = O.direct_disp if kind == "disp" else O.direct_stress
    ref = f(trg, src, nrm, sl, dl, G2, NU2)
    with make_ctx(K, G2, NU2) as c:
        for prec, dt, tol in ((K.KFMM_FP64, torch.float64, 1e-12), (K.KFMM_FP32, torch.float32, 3e-5)):
            out = torch.zeros(nt, no, dtype=dt, device="cuda:0")
            c.direct(dev(trg, dt), dev(src, dt), dev(nrm, dt), None if sl is None else dev(sl, dt),
                     None if dl is None else dev(dl, dt), out, kk, prec)
            assert rel(out.cpu().numpy(), ref) < tol
        # host arrays are accepted too (staged by the library)
        out_h = np.zeros((nt, no))
        c.direct(trg, src, nrm, sl, dl, out_h, kk, K.KFMM_FP64)
        assert rel(out_h, ref) < 1e-12


# ----------------------------------------------------------------- tree and lists
def check_tree(K, c, src, trg, cap):
    tr = c.export_tree()
    st = c.stats()
    nb = st["n_boxes"]
    assert np.array_equal(np.sort(tr["src_perm"]), np.arange(len(src)))
    assert np.array_equal(np.sort(tr["trg_perm"]), np.arange(len(trg)))
    lvl, anc, par = tr["level"], tr["anchor"], tr["parent"]
    U_off, U = c.export_list("U")
    V_off, V = c.export_list("V")
    W_off, Wl = c.export_list("W")
    X_off, X = c.export_list("X")
    children = [[] for _ in range(nb)]
    for b in range(1, nb):
        children[par[b]].append(b)
    leaf = np.array([len(ch) == 0 for ch in children])
    assert leaf.sum() == st["n_leaves"]
    # leaves partition the sorted points; non-leaves hold more than cap points
    for key in ("src", "trg"):
        rng_ = tr[key][leaf]
        rng_ = rng_[np.argsort(rng_[:, 0])]
        lens = rng_[:, 1] - rng_[:, 0]
        assert lens.sum() == (len(src) if key == "src" else len(trg))
        nz = rng_[lens > 0]
        assert np.all(nz[1:, 0] == nz[:-1, 1])
    for b in np.nonzero(~leaf)[0]:
        ns_ = tr["src"][b, 1] - tr["src"][b, 0]
        nt_ = tr["trg"][b, 1] - tr["trg"][b, 0]
        assert max(ns_, nt_) > cap
    # points lie inside their leaf box (geometry from the root cube)
    lo = np.minimum(src.min(0), trg.min(0))
    hi = np.maximum(src.max(0), trg.max(0))
    w = (hi - lo).max() * (1 + 1e-6)
    root_lo = 0.5 * (lo + hi) - 0.5 * w
    ssorted = src[tr["src_perm"]]
    for b in np.nonzero(leaf)[0][:200]:
        s = w / 2 ** lvl[b]
        blo = root_lo + anc[b] * s
        p = ssorted[tr["src"][b, 0]:tr["src"][b, 1]]
        assert np.all(p >= blo - 1e-5 * w) and np.all(p <= blo + s + 1e-5 * w)

    # coverage: every (target leaf, source leaf) pair is counted exactly once
    desc_leaves = {}

    def leaves_under(b):
        if b not in desc_leaves:
            desc_leaves[b] = [b] if leaf[b] else [x for ch in children[b] for x in leaves_under(ch)]
        return desc_leaves[b]

    leaf_ids = np.nonzero(leaf)[0]
    pos = {b: i for i, b in enumerate(leaf_ids)}
    for b in leaf_ids[:: max(1, len(leaf_ids) // 150)]:
        cnt = np.zeros(len(leaf_ids), np.int32)
        for s in U[U_off[b]:U_off[b + 1]]:
            cnt[pos[s]] += 1
        for w_ in Wl[W_off[b]:W_off[b + 1]]:
            for s in leaves_under(w_):
                cnt[pos[s]] += 1
        a = b
        while a >= 0:
            for v in V[V_off[a]:V_off[a + 1]]:
                for s in leaves_under(v):
                    cnt[pos[s]] += 1
            for x in X[X_off[a]:X_off[a + 1]]:
                cnt[pos[x]] += 1
            a = par[a] if a > 0 else -1
        assert np.all(cnt == 1), (b, np.unique(cnt, return_counts=True))
    return st


@pytest.mark.parametrize("cloud", ["surface", "volume", "separate"])
def test_tree_invariants_and_list_coverage(K, cloud):
    cap = 32
    if cloud == "surface":
        src, nrm = W.box_with_voids_points(30000, n_voids=8)
        trg = src
    elif cloud == "volume":
        src, nrm = W.uniform_cloud(20000)
        trg = src
    else:
        src, nrm = W.box_with_voids_points(20000, n_voids=6)
        trg, _ = W.uniform_cloud(7001, lo=(0.05, 0.05, 0.05), hi=(1.95, 0.95, 0.95))
    with make_ctx(K, leaf_cap=cap) as c:
        c.build(dev(src), dev(nrm), dev(trg))
        st = check_tree(K, c, src, trg, cap)
        assert st["n_levels"] >= 3


# ----------------------------------------------------------------- FMM parity
def fmm_case(K, src, nrm, trg, sl, dl, kind, G, nu, p=6, cap=64, nsample=None):
    src, nrm, trg, sl, dl = r32(src), r32(nrm), r32(trg), r32(sl), r32(dl)
    no = 3 if kind == K.KFMM_DISP else 6
    with make_ctx(K, G, nu, p=p, leaf_cap=cap) as c:
        c.build(dev(src), dev(nrm), dev(trg))
        out = torch.zeros(len(trg), no, dtype=torch.float32, device="cuda:0")
        c.eval(None if sl is None else dev(sl), None if dl is None else dev(dl), out, kind)
        got = out.cpu().numpy()
        st = c.stats()
    idx = np.arange(len(trg)) if nsample is None else W.subsample(len(trg), nsample)
    f = O.direct_disp if kind == K.KFMM_DISP else O.direct_stress
    ref = f(trg[idx], src, nrm, sl, dl, G, nu)
    return rel(got[idx], ref), st


@pytest.mark.parametrize("layers", ["sl", "dl", "both"])
def test_fmm_surface_cloud_disp(K, layers):
    src, nrm = W.box_with_voids_points(40000, n_voids=10)
    sl, dl = W.densities(len(src))
    sl = sl if layers in ("sl", "both") else None
    dl = dl if layers in ("dl", "both") else None
    err, st = fmm_case(K, src, nrm, src, sl, dl, K.KFMM_DISP, G1, NU1, nsample=3000)
    assert st["n_v_pairs"] > 0 and st["n_levels"] >= 4
    assert err < 1e-4, err


def test_fmm_volume_cloud_material(K):
    src, nrm = W.uniform_cloud(30011)
    sl, dl = W.densities(len(src))
    err, st = fmm_case(K, src, nrm, src, sl, dl, K.KFMM_DISP, G2, NU2, nsample=3000)
    assert err < 1e-4, err


def test_fmm_separate_targets_stress(K):
    """Stress at volume targets from surface sources (the topological-derivative layout)."""
    src, nrm = W.box_with_voids_points(30000, n_voids=6)
    sl, dl = W.densities(len(src))
    trg, _ = W.uniform_cloud(5003, lo=(0.1, 0.1, 0.1), hi=(1.9, 0.9, 0.9), seed=9)
    err, st = fmm_case(K, src, nrm, trg, sl, dl, K.KFMM_STRESS, G2, NU2, nsample=2000)
    assert err < 1e-4, err


def test_fmm_single_leaf_and_tiny(K):
    """n <= leaf cap: the root is the only box and the sum is all near field."""
    src, nrm = W.uniform_cloud(50)
    sl, dl = W.densities(50)
    err, st = fmm_case(K, src, nrm, src, sl, dl, K.KFMM_DISP, G1, NU1)
    assert st["n_boxes"] == 1 and err < 2e-6
    err, st = fmm_case(K, src[:1], nrm[:1], src[:3] + 0.1, sl[:1], dl[:1], K.KFMM_DISP, G1, NU1)
    assert err < 2e-6


def test_fmm_p_convergence(K):
    src, nrm = W.box_with_voids_points(20000, n_voids=5)
    sl, dl = W.densities(len(src))
    errs = [fmm_case(K, src, nrm, src, sl, dl, K.KFMM_DISP, G1, NU1, p=p, nsample=1500)[0] for p in (4, 5, 6)]
    assert errs[0] < 2e-3 and errs[2] < errs[0] / 3, errs


def test_fmm_errors(K):
    with make_ctx(K) as c:
        x = dev(np.zeros((4, 3)))
        out = torch.zeros(4, 3, device="cuda:0")
        with pytest.raises(K.KfmmError) as e:
            c.eval(x, None, out)
        assert e.value.status == K.KFMM_ERR_NOT_BUILT
        bad = np.zeros((4, 3))
        bad[2, 1] = np.nan
        with pytest.raises(K.KfmmError) as e:
            c.build(dev(bad), None, dev(bad))
        assert e.value.status == K.KFMM_ERR_INVALID_ARG
        c.build(x, None, x)
        with pytest.raises(K.KfmmError) as e:  # double layer without normals
            c.eval(None, x, out)
        assert e.value.status == K.KFMM_ERR_INVALID_ARG


def test_tensor_cores_match_fp32_simt(K):
    """The products on the tcgen05 tensor cores (BF16 split pairs, FP32 accumulation) agree
    with the FP32 SIMT products on the same tree: M2L alone (bit 0), M2L and the box
    operators (bits 0 and 1), neither, and M2L by row tiles of the translation (bits 0 and 4)
    all meet the FMM tolerance against the oracle and differ from each other by the
    split-pair rounding (~1e-5)."""
    src, nrm = W.box_with_voids_points(40000, n_voids=10)
    sl, dl = W.densities(len(src))
    src, nrm, sl, dl = r32(src), r32(nrm), r32(sl), r32(dl)
    outs = []
    for tcores in (3, 1, 0, 17):
        with make_ctx(K, G1, NU1, m2l_tensor_cores=tcores) as c:
            c.build(dev(src), dev(nrm), dev(src))
            out = torch.zeros(len(src), 3, device="cuda:0")
            c.eval(dev(sl), dev(dl), out)
            outs.append(out.cpu().numpy().astype(np.float64))
            assert c.stats()["n_v_pairs"] > 0
    idx = W.subsample(len(src), 2000)
    ref = O.direct_disp(src[idx], src, nrm, sl, dl, G1, NU1)
    for o in outs:
        assert rel(o[idx], ref) < 1e-4
    assert rel(outs[1], outs[2]) < 2e-5
    assert rel(outs[0], outs[2]) < 4e-5
    # M2L with the pairs as rows (1) and by row tiles of the translation (17): the same split
    # products summed in another order
    assert rel(outs[3], outs[2]) < 2e-5
    assert rel(outs[1], outs[3]) < 1e-5


def test_graph_replay_matches_and_invalidates(K):
    """Repeated evaluations with the same arguments are captured into a CUDA graph and replayed;
    the replayed results equal a plain evaluation (up to the order of the reductions), and a
    new build or material drops the graph."""
    src, nrm = W.box_with_voids_points(30000, n_voids=10)
    sl, dl = W.densities(len(src))
    src, nrm, sl, dl = r32(src), r32(nrm), r32(sl), r32(dl)
    x, n, s, d = dev(src), dev(nrm), dev(sl), dev(dl)
    out = torch.zeros(len(src), 3, device="cuda:0")
    with make_ctx(K, G1, NU1, graphs=0) as c:
        c.build(x, n, x)
        c.eval(s, d, out)
        ref = out.cpu().numpy().astype(np.float64)
    with make_ctx(K, G1, NU1) as c:
        c.build(x, n, x)
        res, launches = [], []
        for _ in range(4):
            l0 = c.stats()["kernel_launches"]
            out.zero_()
            c.eval(s, d, out)
            res.append(out.cpu().numpy().astype(np.float64))
            launches.append(c.stats()["kernel_launches"] - l0)
        for r_ in res:
            assert rel(r_, ref) < 1e-5
        # the first call also makes the plans; every later one (plain, captured, replayed)
        # launches the same kernels, which the graph counts
        assert launches[1] > 10 and len(set(launches[1:])) == 1 and launches[0] >= launches[1]
        # a new set of points: the graph must not replay the old tree
        src2 = r32(src * 0.5 + 0.25)
        c.build(dev(src2), n, dev(src2))
        out.zero_()
        c.eval(s, d, out)
        idx = W.subsample(len(src), 500)
        ref2 = O.direct_disp(src2[idx], src2, nrm, sl, dl, G1, NU1)
        assert rel(out.cpu().numpy().astype(np.float64)[idx], ref2) < 1e-4


@pytest.mark.parametrize("kind", ["disp", "stress"])
def test_density_columns_batched(K, kind):
    """ncol density columns evaluated in one pass (every phase over all columns) equal the
    columns evaluated one by one, and the oracle."""
    src, nrm = W.box_with_voids_points(25000, n_voids=10)
    ncol = 3
    sl, dl = W.densities(len(src), ncol=ncol)
    src, nrm, sl, dl = r32(src), r32(nrm), r32(sl), r32(dl)
    kd = K.KFMM_DISP if kind == "disp" else K.KFMM_STRESS
    no = 3 if kind == "disp" else 6
    cfg = {} if kind == "disp" else dict(p=8, m2l_rtol=1e-7)
    with make_ctx(K, G1, NU1, **cfg) as c:
        c.build(dev(src), dev(nrm), dev(src))
        out = torch.zeros(len(src), no * ncol, device="cuda:0")
        c.eval(dev(sl), dev(dl), out, kind=kd, ncol=ncol)
        batched = out.cpu().numpy().astype(np.float64)
        one = torch.zeros(len(src), no, device="cuda:0")
        for col in range(ncol):
            s1 = np.ascontiguousarray(sl[:, 3 * col:3 * col + 3])
            d1 = np.ascontiguousarray(dl[:, 3 * col:3 * col + 3])
            c.eval(dev(s1), dev(d1), one, kind=kd)
            ref = one.cpu().numpy().astype(np.float64)
            assert rel(batched[:, no * col:no * col + no], ref) < 2e-6
    idx = W.subsample(len(src), 300)
    fn = O.direct_disp if kind == "disp" else O.direct_stress
    tol = 1e-4 if kind == "disp" else 5e-4
    for col in range(ncol):
        s1 = np.ascontiguousarray(sl[:, 3 * col:3 * col + 3])
        d1 = np.ascontiguousarray(dl[:, 3 * col:3 * col + 3])
        ref = fn(src[idx], src, nrm, s1, d1, G1, NU1)
        assert rel(batched[idx, no * col:no * col + no], ref) < tol


def test_autotuned_launch_shapes(K):
    """The first evaluation picks the M2L chunk and the leaf-item cost cap among its
    candidates by timing them on the tree; the result does not depend on the choice."""
    src, nrm = W.box_with_voids_points(60000, n_voids=10)
    sl, dl = W.densities(len(src))
    src, nrm, sl, dl = r32(src), r32(nrm), r32(sl), r32(dl)
    outs = []
    for tune in (0, 1):
        with make_ctx(K, G1, NU1, autotune=tune) as c:
            c.build(dev(src), dev(nrm), dev(src))
            out = torch.zeros(len(src), 3, device="cuda:0")
            c.eval(dev(sl), dev(dl), out)
            st = c.stats()
            outs.append(out.cpu().numpy().astype(np.float64))
            if tune:
                assert st["m2l_chunk"] in (256, 512, 1024, 2048)
                assert st["eval_item_cost"] in (256.0, 512.0, 1024.0, 2048.0, 4096.0)
                c.eval(dev(sl), dev(dl), out)  # tuned shapes kept, same answer
                assert rel(out.cpu().numpy().astype(np.float64), outs[0]) < 1e-5
            else:
                assert st["m2l_chunk"] == 1024 and st["eval_item_cost"] == 1024.0
    assert rel(outs[1], outs[0]) < 1e-5


@pytest.mark.parametrize("kind", ["disp", "stress"])
def test_overlapped_streams_match_one_stream(K, kind):
    """With the near field (P2L and the leaf-to-leaf P2P) on the second stream, concurrent
    with the upward pass and M2L, the result equals the one-stream evaluation up to the order
    of the atomic sums, for plain calls, graph replays and profiled (serialised) calls."""
    src, nrm = W.box_with_voids_points(50000, n_voids=10)
    ncol = 2
    sl, dl = W.densities(len(src), ncol=ncol)
    src, nrm, sl, dl = r32(src), r32(nrm), r32(sl), r32(dl)
    kd = K.KFMM_DISP if kind == "disp" else K.KFMM_STRESS
    no = (3 if kind == "disp" else 6) * ncol
    x, n, s, d = dev(src), dev(nrm), dev(sl), dev(dl)
    cfg = {} if kind == "disp" else dict(p=8, m2l_rtol=1e-7)
    res = {}
    for streams in (0, 1):
        with make_ctx(K, G1, NU1, streams=streams, **cfg) as c:
            c.build(x, n, x)
            outs = []
            for k in range(4):  # plain, plain, captured, replayed
                out = torch.full((len(src), no), float("nan"), device="cuda:0")
                c.eval(s, d, out, kind=kd, ncol=ncol)
                outs.append(out.cpu().numpy().astype(np.float64))
            c.set_profiling(True)
            out = torch.full((len(src), no), float("nan"), device="cuda:0")
            c.eval(s, d, out, kind=kd, ncol=ncol)
            outs.append(out.cpu().numpy().astype(np.float64))
            c.set_profiling(False)
            res[streams] = outs
    for o in res[0] + res[1]:
        assert np.all(np.isfinite(o))
        assert rel(o, res[0][0]) < 1e-5
    idx = W.subsample(len(src), 300)
    fn = O.direct_disp if kind == "disp" else O.direct_stress
    tol = 1e-4 if kind == "disp" else 5e-4
    s1, d1 = np.ascontiguousarray(sl[:, 3:6]), np.ascontiguousarray(dl[:, 3:6])
    ref = fn(src[idx], src, nrm, s1, d1, G1, NU1)
    assert rel(res[1][3][idx, no // 2:], ref) < tol


@pytest.mark.parametrize("p", [4, 6])
def test_leaf_items_every_cost_and_split(K, p):
    """The leaf-evaluation work items cover every (target chunk, source segment) once for every
    item cost cap, with the near / far lists split (streams 1) or one list (streams 0): the
    results agree with each other and with the oracle.  Small caps cut many items per chunk
    (p = 4 puts most W boxes through their upward densities)."""
    src, nrm = W.box_with_voids_points(20000, n_voids=5)
    sl, dl = W.densities(len(src))
    src, nrm, sl, dl = r32(src), r32(nrm), r32(sl), r32(dl)
    x, n, s, d = dev(src), dev(nrm), dev(sl), dev(dl)
    idx = W.subsample(len(src), 600)
    ref = O.direct_disp(src[idx], src, nrm, sl, dl, G1, NU1)
    outs = []
    for cost in (64, 256, 1024, 4096):
        for streams in (0, 1):
            with make_ctx(K, G1, NU1, p=p, streams=streams, eval_item_cost=cost) as c:
                c.build(x, n, x)
                out = torch.full((len(src), 3), float("nan"), device="cuda:0")
                c.eval(s, d, out)
                assert c.stats()["eval_item_cost"] == float(cost)
                outs.append(out.cpu().numpy().astype(np.float64))
    tol = 3e-3 if p == 4 else 1e-4
    for o in outs:
        assert np.all(np.isfinite(o))
        assert rel(o[idx], ref) < tol
        assert rel(o, outs[0]) < 1e-5


def _point_sets(sizes, seed0=11):
    """Uneven box-with-voids surfaces, each scaled and shifted; sets 0 and 1 overlap in space
    (no interaction may cross sets even where their points interleave)."""
    pts, nrm = [], []
    for k, n in enumerate(sizes):
        x, nn = W.box_with_voids_points(n, n_voids=3 + k, seed=seed0 + k)
        scale = 1.0 + 0.5 * k
        shift = np.array([0.0, 0.0, 0.0]) if k < 2 else np.array([3.0 * k, -1.0 * k, 0.5])
        pts.append(x * scale + shift)
        nrm.append(nn)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    return np.concatenate(pts), np.concatenate(nrm), off


@pytest.mark.parametrize("kind", ["disp", "stress"])
def test_point_sets_one_build(K, kind):
    """kfmm_build_sets: several independent surfaces of uneven size in one tree and one set of
    launches.  Each set's result equals its own build (the per-set trees are the same) and
    the oracle restricted to the set."""
    sizes = [6000, 2500, 700, 9000]
    src, nrm, off = _point_sets(sizes)
    ncol = 2
    sl, dl = W.densities(len(src), ncol=ncol)
    src, nrm, sl, dl = r32(src), r32(nrm), r32(sl), r32(dl)
    kd = K.KFMM_DISP if kind == "disp" else K.KFMM_STRESS
    no = (3 if kind == "disp" else 6) * ncol
    cfg = {} if kind == "disp" else dict(p=8, m2l_rtol=1e-7)
    with make_ctx(K, G1, NU1, **cfg) as c:
        c.build_sets(off, dev(src), dev(nrm), off, dev(src))
        st = c.stats()
        out = torch.full((len(src), no), float("nan"), device="cuda:0")
        c.eval(dev(sl), dev(dl), out, kind=kd, ncol=ncol)
        batched = out.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(batched))
        nb_sum = 0
        for k in range(len(sizes)):
            a, b = off[k], off[k + 1]
            c.build(dev(src[a:b]), dev(nrm[a:b]), dev(src[a:b]))
            nb_sum += c.stats()["n_boxes"]
            one = torch.zeros(b - a, no, device="cuda:0")
            c.eval(dev(sl[a:b]), dev(dl[a:b]), one, kind=kd, ncol=ncol)
            assert rel(batched[a:b], one.cpu().numpy().astype(np.float64)) < 2e-6
        assert st["n_boxes"] == nb_sum  # the forest is the union of the per-set trees
    fn = O.direct_disp if kind == "disp" else O.direct_stress
    tol = 1e-4 if kind == "disp" else 5e-4
    for k in (0, 1, 3):
        a, b = off[k], off[k + 1]
        idx = a + W.subsample(b - a, 150)
        s1, d1 = np.ascontiguousarray(sl[a:b, 3:6]), np.ascontiguousarray(dl[a:b, 3:6])
        ref = fn(src[idx], src[a:b], nrm[a:b], s1, d1, G1, NU1)
        assert rel(batched[idx, no // 2:], ref) < tol


def test_point_sets_separate_targets_and_errors(K):
    """Sets with their own target points; bad offsets are refused."""
    sizes = [3000, 5000, 1200]
    src, nrm, off = _point_sets(sizes, seed0=21)
    trg_sizes = [400, 900, 300]
    trg = np.concatenate([src[off[k]:off[k + 1]][W.subsample(sizes[k], trg_sizes[k])] * 0.97 + 0.01
                          for k in range(3)])
    toff = np.concatenate([[0], np.cumsum(trg_sizes)]).astype(np.int64)
    sl, dl = W.densities(len(src))
    src, nrm, trg, sl, dl = r32(src), r32(nrm), r32(trg), r32(sl), r32(dl)
    with make_ctx(K, G1, NU1) as c:
        c.build_sets(off, dev(src), dev(nrm), toff, dev(trg))
        out = torch.zeros(len(trg), 3, device="cuda:0")
        c.eval(dev(sl), dev(dl), out)
        got = out.cpu().numpy().astype(np.float64)
        for k in range(3):
            ref = O.direct_disp(trg[toff[k]:toff[k + 1]], src[off[k]:off[k + 1]], nrm[off[k]:off[k + 1]],
                                sl[off[k]:off[k + 1]], dl[off[k]:off[k + 1]], G1, NU1)
            assert rel(got[toff[k]:toff[k + 1]], ref) < 1e-4
        bad = off.copy()
        bad[2] = bad[1]  # an empty set
        with pytest.raises(K.KfmmError):
            c.build_sets(bad, dev(src), dev(nrm), toff, dev(trg))


def test_clustered_points_deep_tree(K):
    """A tight cluster inside a unit cloud needs more than the 10 levels the keys are first
    made with: the build goes back to full-depth keys, and the FMM still meets its tolerance.
    The cluster sits near the origin, where FP32 positions resolve its smallest boxes (a box
    whose half-width is near the FP32 spacing of its coordinates misplaces its check and
    equivalent surfaces)."""
    rng = np.random.default_rng(5)
    far, nf = W.uniform_cloud(6000)
    near = 1e-3 + 1e-4 * rng.uniform(-1.0, 1.0, size=(6000, 3))
    nn = rng.normal(size=(6000, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    src = r32(np.concatenate([far, near]))
    nrm = r32(np.concatenate([nf, nn]))
    sl, dl = W.densities(len(src))
    sl, dl = r32(sl), r32(dl)
    with make_ctx(K, G1, NU1) as c:
        c.build(dev(src), dev(nrm), dev(src))
        st = c.stats()
        assert st["n_levels"] > 11
        # deepest half-width over the FP32 spacing at the root cube's largest coordinate
        half = 0.5 / 2.0 ** (st["n_levels"] - 1)
        assert 0.4 * half * 2.0 ** 23 <= st["fp32_box_ratio"] <= 2.5 * half * 2.0 ** 23
        out = torch.zeros(len(src), 3, device="cuda:0")
        c.eval(dev(sl), dev(dl), out)
        got = out.cpu().numpy().astype(np.float64)
    idx = np.concatenate([W.subsample(6000, 150), 6000 + W.subsample(6000, 150)])
    ref = O.direct_disp(src[idx], src, nrm, sl, dl, G1, NU1)
    assert rel(got[idx], ref) < 1e-4


def test_full_size_bench_workload(K):
    """The benchmark workload at its full size and in the launch configuration the benchmark
    times (1e6 surface points of the box with 20 voids, p = 6, leaf cap 64, tuned launch
    shapes, overlapped streams): 300 sampled targets against the oracle, one by one."""
    n = 1_000_000
    src, nrm = W.box_with_voids_points(n, n_voids=20)
    sl, dl = W.densities(n)
    src, nrm, sl, dl = r32(src), r32(nrm), r32(sl), r32(dl)
    with make_ctx(K, G1, NU1, p=6, leaf_cap=64) as c:
        x = dev(src)
        c.build(x, dev(nrm), x)
        out = torch.full((n, 3), float("nan"), device="cuda:0")
        c.eval(dev(sl), dev(dl), out)
        got = out.cpu().numpy().astype(np.float64)
        st = c.stats()
        assert st["n_levels"] >= 8
        assert st["fp32_box_ratio"] > 1000  # FP32 positions resolve the deepest boxes
    assert np.all(np.isfinite(got))
    idx = W.subsample(n, 300)
    ref = O.direct_disp(src[idx], src, nrm, sl, dl, G1, NU1)
    assert rel(got[idx], ref) < 1e-4


def test_bounded_wait_gives_up_and_context_survives(K):
    """Failure detection without a GPU fault: a device wait on a barrier that nothing
    arrives on gives up after its poll limit, the time-out reaches the host as
    KFMM_ERR_DEVICE_TIMEOUT through the device error word, and the context keeps working."""
    src, nrm = W.box_with_voids_points(4000, n_voids=3)
    sl, dl = W.densities(len(src))
    src, nrm, sl, dl = r32(src), r32(nrm), r32(sl), r32(dl)
    with make_ctx(K, G1, NU1) as c:
        assert c.selftest_bounded_wait(4096) == K.KFMM_ERR_DEVICE_TIMEOUT
        assert "as designed" in K._lib.kfmm_last_error(c.handle).decode()
        c.build(dev(src), dev(nrm), dev(src))
        out = torch.zeros(len(src), 3, device="cuda:0")
        c.eval(dev(sl), dev(dl), out)
        idx = W.subsample(len(src), 200)
        ref = O.direct_disp(src[idx], src, nrm, sl, dl, G1, NU1)
        assert rel(out.cpu().numpy().astype(np.float64)[idx], ref) < 1e-4


def test_contexts_of_different_rank_coexist(K):
    """Two contexts whose M2L ranks differ (different basis cuts) alternate evaluations: the
    shared-memory limit of a tensor-core kernel belongs to the function, so building the
    smaller context must not shrink it below what the larger one launches with."""
    src, nrm = W.box_with_voids_points(20000, n_voids=6)
    sl, dl = W.densities(len(src))
    src, nrm, sl, dl = r32(src), r32(nrm), r32(sl), r32(dl)
    idx = W.subsample(len(src), 200)
    ref = O.direct_disp(src[idx], src, nrm, sl, dl, G1, NU1)
    with make_ctx(K, G1, NU1) as a, make_ctx(K, G1, NU1, m2l_rtol=1e-3) as b:
        outs = {}
        for name, c in (("a", a), ("b", b), ("a2", a)):
            if name != "a2":
                c.build(dev(src), dev(nrm), dev(src))
            out = torch.zeros(len(src), 3, device="cuda:0")
            c.eval(dev(sl), dev(dl), out)
            outs[name] = out.cpu().numpy().astype(np.float64)
        assert b.stats()["m2l_rank"] < a.stats()["m2l_rank"]
    assert rel(outs["a"][idx], ref) < 1e-4
    assert rel(outs["a2"], outs["a"]) < 1e-6
    assert rel(outs["b"][idx], ref) < 1e-2
