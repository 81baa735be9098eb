"""The compensated all-pairs displacement sum (kfmm_direct_hi) and the mixed-precision GMRES
that uses it as its outer operator (Sec. "Numerical solution": GMRES on Eq. num2).

The sum must be FP64-grade where FP32 errors would not average out: a GMRES residual b - A x
on a clamped cantilever cancels by ||A| |x|| / ||b|| ~ 100 (measured with the oracle's dense
system), so the operator has to be right to ~1e-9 of its terms for a 1e-6 residual to mean
anything.  What remains is the random rounding of the FP32 pairs beyond the near radius,
~4e-7 of the root sum of squares of their terms (falling as 1 / near radius).  Tolerances:
 - against the GPU FP64 direct sum, near radius 4 edges, on the densities of a rigid
   rotation and of a cantilever solution (smooth densities, as in a solve): 5e-8 relative L2
   and 20x closer than the plain FP32 sum (measured 2.1e-8 against 1.3e-6); on random
   densities (no structure; each term's rounding shows): no worse than the plain FP32 sum
   and within 1e-6 (measured 4.3e-7);
 - M(u, t) of the BEM operator (near radius 4 edges) on a cantilever solution: within 1e-6
   of ||b|| of the FP64 operator (the budget of a 1e-6 residual);
 - a 51,840-triangle cantilever, GMRES-IR to 2e-7 in the compensated operator's residual:
   at sampled rows the operator differs from the CPU oracle's by less than 8e-7 of ||b||
   (measured 4.9e-7 with a near radius of 16 edges, 7.8e-7 of the FP64 sum at 4), and the
   oracle's residual of the solution is below 1e-6 of ||b|| (the triangle inequality:
   2e-7 + 8e-7).
"""
import time

import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

G0, NU0 = 1.0, 0.3


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_04082_gb300 as K
    return K


def quad_sources(V, T):
    nrm, area, cen = O.tri_geometry(V, T)
    q, w = O.tri_quadrature(V, T)
    q[12::16] = cen  # the centre sub-triangle's centroid is the collocation point itself
    return q, w, np.repeat(nrm, 16, axis=0), nrm, area, cen


def test_direct_hi_matches_fp64_direct_on_cancelling_densities(K):
    """Rigid rotation u = w x y on a closed box (1/2 u + P u = 0 in the continuum, so the sum
    is cancelled by 1/2 u in the operator) and the cantilever's dense solution, near radius
    4 edges: the compensated sum agrees with the FP64 sum to 5e-8 relative L2, at least 20
    times closer than the plain FP32 sum."""
    V, T, mask, vals = W.cantilever(6)[:4]
    q, w, qn, nrm, area, cen = quad_sources(V, T)
    H, Gm = O.bem_assemble(V, T, G0, NU0)
    A, bb = O.bem_system(H, Gm, mask, vals)
    u_sol, t_sol = O.unknowns_to_fields(np.linalg.solve(A, bb), mask, vals)
    omega = np.array([0.3, -1.1, 0.7])
    cases = {"rotation": (np.cross(omega, cen), np.zeros_like(cen)), "cantilever": (u_sol, t_sol)}
    dev = "cuda"
    with K.Kfmm() as f:
        f.set_material(K.material_K(G0, NU0), G0)
        for name, (u, t) in cases.items():
            sl = -np.repeat(t, 16, axis=0) * w[:, None]
            dl = np.repeat(u, 16, axis=0) * w[:, None]
            args = [torch.tensor(a, dtype=torch.float64, device=dev) for a in (cen, q, qn, sl, dl)]
            hi = torch.zeros(len(cen), 3, dtype=torch.float64, device=dev)
            ref = torch.zeros_like(hi)
            f32 = torch.zeros(len(cen), 3, dtype=torch.float32, device=dev)
            f.direct_hi(*args, hi, near_radius=4 / 6)  # 4 x the longest edge (the voxel size)
            f.direct(*args, ref, K.KFMM_DISP, K.KFMM_FP64)
            f.direct(*[a.float() for a in args], f32, K.KFMM_DISP, K.KFMM_FP32)
            torch.cuda.synchronize()
            hi, ref, f32 = (x.double().cpu().numpy() for x in (hi, ref, f32))
            e_hi = np.linalg.norm(hi - ref) / np.linalg.norm(ref)
            e_32 = np.linalg.norm(f32 - ref) / np.linalg.norm(ref)
            print(f"{name}: compensated {e_hi:.2e}, plain FP32 {e_32:.2e}")
            assert e_hi < 5e-8, (name, e_hi)
            assert e_hi < e_32 / 20, (name, e_hi, e_32)


def test_direct_hi_random_and_arguments(K):
    """Random points and densities, SL-only, DL-only and SL+DL, near radius 0 and > 0: within the
    FP32 kernel rounding of the FP64 sum (1e-6 relative L2) and no worse than the plain FP32
    sum; host arrays are staged; bad arguments are rejected."""
    rng = np.random.default_rng(5)
    ns, nt = 7001, 1537
    src = rng.uniform(-1, 1, (ns, 3)) + 3.0  # away from the origin: hi/lo splitting matters
    trg = np.concatenate([rng.uniform(-1, 1, (nt - 5, 3)) + 3.0, src[:5]])  # 5 coincident points
    nrm = rng.normal(size=(ns, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    sl, dl = rng.normal(size=(ns, 3)), rng.normal(size=(ns, 3))
    with K.Kfmm() as f:
        f.set_material(K.material_K(1.7, 0.27), 1.7)
        for s_, d_ in ((sl, dl), (sl, None), (None, dl)):
            ref = np.zeros((nt, 3))
            f.direct(trg, src, nrm, s_, d_, ref, K.KFMM_DISP, K.KFMM_FP64)
            f32 = np.zeros((nt, 3), np.float32)
            f.direct(*(None if a is None else a.astype(np.float32) for a in (trg, src, nrm, s_, d_)), f32,
                     K.KFMM_DISP, K.KFMM_FP32)
            e32 = np.linalg.norm(f32 - ref) / np.linalg.norm(ref)
            for rad in (0.0, 0.3):
                out = np.zeros((nt, 3))
                f.direct_hi(trg, src, nrm, s_, d_, out, near_radius=rad)  # host arrays
                e = np.linalg.norm(out - ref) / np.linalg.norm(ref)
                assert e < 1e-6 and e <= e32, (e, e32)
        out = np.zeros((nt, 3))
        for bad in ({"near_radius": -1.0}, {"near_radius": float("nan")}):
            with pytest.raises(K.KfmmError) as e:
                f.direct_hi(trg, src, nrm, sl, dl, out, **bad)
            assert e.value.status == K.KFMM_ERR_INVALID_ARG
        with pytest.raises(K.KfmmError) as e:
            f.direct_hi(trg, src, None, sl, dl, out)  # double layer without normals
        assert e.value.status == K.KFMM_ERR_INVALID_ARG


@pytest.mark.parametrize("refine,tol", [(1, 1e-6), (2, 1e-8)])
def test_gmres_ir_outer_operators_agree(K, refine, tol):
    """GMRES-IR with the compensated outer operator (refine = 1, to 1e-6) and with the FP64
    direct one (refine = 2, to 1e-8): the residual of the oracle's dense system is within
    twice the tolerance, and the solution matches the dense one."""
    V, T, mask, vals = W.cantilever(4)[:4]
    H, Gm = O.bem_assemble(V, T, G0, NU0)
    A, bb = O.bem_system(H, Gm, mask, vals)
    u_ref, t_ref = O.unknowns_to_fields(np.linalg.solve(A, bb), mask, vals)
    with K.Bem(V, T, K.BEM_FMM) as b:
        b.set_material(K.material_K(G0, NU0), G0)
        b.set_bc(mask, vals)
        u, t = np.zeros((len(T), 3)), np.zeros((len(T), 3))
        st = b.solve(u, t, tol=tol, restart=100, maxit=3000, refine=refine, inner_tol=1e-3)
    assert st["converged"] and st["relres"] <= tol
    assert st["matvecs_hi"] == st["outer"] + 1
    x = np.where(mask.reshape(-1) > 0, t.reshape(-1), u.reshape(-1))
    assert np.linalg.norm(A @ x - bb) / np.linalg.norm(bb) < 2 * tol
    rel = lambda a, r: np.linalg.norm(a - r) / np.linalg.norm(r)  # noqa: E731
    assert rel(u, u_ref) < 100 * tol and rel(t, t_ref) < 1000 * tol


def test_bem_operator_direct_hi_matches_fp64(K):
    """The BEM operator built on the compensated sum (BEM_DIRECT_HI) against the FP64 one:
    M(u, t) of the cantilever solution agrees to 1e-6 of ||b||."""
    V, T, mask, vals = W.cantilever(6)[:4]
    H, Gm = O.bem_assemble(V, T, G0, NU0)
    A, bb = O.bem_system(H, Gm, mask, vals)
    u, t = O.unknowns_to_fields(np.linalg.solve(A, bb), mask, vals)
    outs = {}
    for op in (K.BEM_DIRECT_HI, K.BEM_DIRECT_FP64):
        with K.Bem(V, T, op) as b:
            b.set_material(K.material_K(G0, NU0), G0)
            o = np.zeros((len(T), 3))
            b.apply(u, t, o)
            outs[op] = o
    e = np.linalg.norm(outs[K.BEM_DIRECT_HI] - outs[K.BEM_DIRECT_FP64]) / np.linalg.norm(bb)
    print(f"|M_hi - M_fp64| / |b| = {e:.2e}")
    assert e < 1e-6


def test_cantilever_52k_gmres_ir_against_oracle_rows(K):
    """Config-3 geometry at 51,840 triangles (voxel h = 1/36, patch 0.25): GMRES-IR with the
    compensated outer operator to 2e-7; then the oracle evaluates M(u, t) = 1/2 u + P^D u -
    U^D t of Eq. num at 200 sampled collocation points (direct sum over all 829,440
    quadrature sources, the element's own terms replaced by its analytic blocks)."""
    n = 36
    V, T, mask, vals = W.cantilever(n)[:4]
    nt = len(T)
    q, w, qn, nrm, area, cen = quad_sources(V, T)
    with K.Bem(V, T, K.BEM_FMM) as b:
        b.set_material(K.material_K(G0, NU0), G0)
        b.set_bc(mask, vals)
        u, t = np.zeros((nt, 3)), np.zeros((nt, 3))
        st = b.solve(u, t, tol=2e-7, restart=100, maxit=4000, refine=1, inner_tol=1e-3)
        assert st["converged"] and st["relres"] <= 2e-7
        rhs = np.zeros((nt, 3))
        b.rhs(rhs)
    with K.Bem(V, T, K.BEM_DIRECT_HI) as b:
        b.set_material(K.material_K(G0, NU0), G0)
        m_hi = np.zeros((nt, 3))
        b.apply(u, t, m_hi)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.apply(u, t, m_hi)
        t_hi = time.perf_counter() - t0
    bn = np.linalg.norm(rhs)
    idx = W.subsample(nt, 200)
    # the oracle's rows: all quadrature sources (own centre point skipped at r = 0), minus the
    # element's own 15 other points, plus its analytic singular blocks
    sl = -np.repeat(t, 16, axis=0) * w[:, None]
    dl = np.repeat(u, 16, axis=0) * w[:, None]
    m_or = O.direct_disp(cen[idx], q, qn, sl, dl, G0, NU0)
    for r, l in enumerate(idx):
        own = slice(16 * l, 16 * l + 16)
        m_or[r] -= O.direct_disp(cen[l:l + 1], q[own], qn[own], sl[own], dl[own], G0, NU0)[0]
        Us, Ts = O.self_integrals(*V[T[l]], G0, NU0)
        m_or[r] += 0.5 * u[l] + Ts @ u[l] - Us @ t[l]
    scale = np.sqrt(len(idx) / nt) * bn  # ||b|| restricted to a uniform sample of the rows
    diff = np.linalg.norm(m_hi[idx] - m_or) / scale
    res = np.linalg.norm(m_or) / scale
    print(f"52k cantilever: |M_hi - M_oracle| = {diff:.2e}, oracle residual {res:.2e} of ||b||, "
          f"{st['iters']} inner iterations, {st['outer']} outer, {st['seconds']:.2f} s per solve, "
          f"compensated operator {1e3 * t_hi:.0f} ms")
    assert diff < 8e-7
    assert res < 1e-6


def test_arrays_of_another_gpu_are_rejected(K):
    """Every entry point refuses device memory of a GPU other than its context's (a kernel
    would otherwise read it without peer access); the check runs before any launch, on the
    pointer attributes alone.  Needs two GPUs."""
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    other = torch.device("cuda", 1)
    trg = torch.zeros(8, 3, dtype=torch.float64, device=other)
    src = torch.ones(8, 3, dtype=torch.float64, device=other)
    out = torch.zeros(8, 3, dtype=torch.float64, device=other)
    with K.Kfmm(device=0) as f:
        for call in (lambda: f.direct(trg, src, None, src, None, out, K.KFMM_DISP, K.KFMM_FP64),
                     lambda: f.direct_hi(trg, src, None, src, None, out),
                     lambda: K.kfmm_direct_noalloc(f.handle, trg, src, None, src, None, out, K.KFMM_DISP,
                                                   K.KFMM_FP64)):
            with pytest.raises(K.KfmmError) as e:
                call()
            assert e.value.status == K.KFMM_ERR_INVALID_ARG
