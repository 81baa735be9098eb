"""Several load cases in one BEM solve (the six unit macro strains of a periodic-cell
homogenisation, Sec. "Periodic cell of a metamaterial": the fluctuation field of each has
the traction t = -sigma^h n on the void surfaces), and the topological-derivative output kind
of the FMM evaluation (Eq. deriv).

Workload: one spherical cavity (radius 0.4, 1280 triangles, normals out of the material,
i.e. into the void) in an infinite medium, G = 1.3, nu = 0.27.  Tolerances: each column of
the 6-column solve matches the oracle's dense solve of that column to 1e-5 relative L2 (the
GMRES tolerance is 1e-7 in the FP64-grade residual) and the same column solved alone to
1e-6; the hydrostatic combination matches the closed form u_r = S a / (4 G) on the wall
within the 1280-triangle discretisation error (1.9%, measured by the oracle's own test);
interior stresses and D^T of all columns at once match the oracle to 1e-4 (the FMM's
tolerance at its interior order).
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

A_CAV, G0, NU0 = 0.4, 1.3, 0.27


@pytest.fixture(scope="module")
def K():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_04082_gb300 as K
    return K


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def unit_strain_tractions(nrm, G, nu):
    """t = -sigma^h n for the 6 unit macro strains (xx, yy, zz, yz, xz, xy), [nt, 18]."""
    lam = 2 * G * nu / (1 - 2 * nu)
    pairs = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    cols = []
    for i, j in pairs:
        eps = np.zeros((3, 3))
        eps[i, j] = eps[j, i] = 1.0 if i == j else 0.5
        sig = lam * np.trace(eps) * np.eye(3) + 2 * G * eps
        cols.append(-nrm @ sig.T)
    return np.concatenate(cols, axis=1)


@pytest.fixture(scope="module")
def cavity():
    V, T = W.icosphere(3, radius=A_CAV, inward=True)
    nrm, area, cen = O.tri_geometry(V, T)
    vals = unit_strain_tractions(nrm, G0, NU0)
    mask = np.zeros((len(T), 3), np.uint8)
    H, Gm = O.bem_assemble(V, T, G0, NU0)
    # all-traction conditions: A = H, b = Gm t per column (Eq. num2 with every u unknown)
    u_ref = np.linalg.solve(H, Gm @ vals.reshape(len(T), 6, 3).transpose(0, 2, 1).reshape(3 * len(T), 6))
    u_ref = u_ref.reshape(len(T), 3, 6).transpose(0, 2, 1).reshape(len(T), 18)
    return V, T, nrm, cen, mask, vals, u_ref


def test_six_load_cases_in_one_solve(K, cavity):
    V, T, nrm, cen, mask, vals, u_ref = cavity
    nt = len(T)
    with K.Bem(V, T, K.BEM_FMM) as b:
        b.set_material(K.material_K(G0, NU0), G0)
        b.set_bc(mask, vals)
        u, t = np.zeros((nt, 18)), np.zeros((nt, 18))
        st = b.solve(u, t, tol=1e-7, restart=60, maxit=2000, refine=1, inner_tol=1e-3)
        assert st["converged"] and st["relres"] <= 1e-7
        assert np.allclose(t, vals)  # the tractions are the prescribed ones
        for c in range(6):
            assert rel(u[:, 3 * c:3 * c + 3], u_ref[:, 3 * c:3 * c + 3]) < 1e-5, c
        # the same columns one at a time
        for c in (0, 4):
            b.set_bc(mask, np.ascontiguousarray(vals[:, 3 * c:3 * c + 3]))
            u1, t1 = np.zeros((nt, 3)), np.zeros((nt, 3))
            b.solve(u1, t1, tol=1e-7, restart=60, maxit=2000, refine=1, inner_tol=1e-3)
            assert rel(u[:, 3 * c:3 * c + 3], u1) < 1e-6, c
    # hydrostatic unit strain = sum of the three normal cases: u_r = S a / (4 G), S = 3 K
    Kb = 2 * G0 * (1 + NU0) / (3 * (1 - 2 * NU0))
    uh = u[:, 0:3] + u[:, 3:6] + u[:, 6:9]
    er = cen / np.linalg.norm(cen, axis=1)[:, None]
    ur = np.einsum("ij,ij->i", uh, er)
    assert np.abs(ur / (3 * Kb * A_CAV / (4 * G0)) - 1).max() < 0.03


def test_multicolumn_plain_gmres_and_rhs(K, cavity):
    """Plain GMRES on the FMM operator (no refinement) for 6 columns, and the right-hand side
    B y of all columns against the oracle's Gm t."""
    V, T, nrm, cen, mask, vals, u_ref = cavity
    nt = len(T)
    H, Gm = O.bem_assemble(V, T, G0, NU0)
    with K.Bem(V, T, K.BEM_FMM) as b:
        b.set_material(K.material_K(G0, NU0), G0)
        b.set_bc(mask, vals[:, :18])
        rhs = np.zeros((nt, 18))
        b.rhs(rhs)
        for c in range(6):
            ref = Gm @ vals[:, 3 * c:3 * c + 3].reshape(-1)
            assert rel(rhs[:, 3 * c:3 * c + 3].reshape(-1), ref) < 1e-4
        u = np.zeros((nt, 18))
        st = b.solve(u, None, tol=1e-5, restart=60, maxit=2000)
        assert st["converged"]
        for c in range(6):
            assert rel(u[:, 3 * c:3 * c + 3], u_ref[:, 3 * c:3 * c + 3]) < 1e-4, c


def test_multicolumn_interior_stress_and_td(K, cavity):
    """Stress and D^T of the 6 stored load cases at material points around the cavity, one
    interior evaluation for all columns, against the oracle per column."""
    V, T, nrm, cen, mask, vals, u_ref = cavity
    rng = np.random.default_rng(9)
    d = rng.normal(size=(300, 3))
    pts = (d / np.linalg.norm(d, axis=1)[:, None] * rng.uniform(1.5, 3.0, (300, 1)) * A_CAV).astype(np.float32)
    with K.Bem(V, T, K.BEM_FMM) as b:
        b.set_material(K.material_K(G0, NU0), G0)
        b.set_solution(u_ref, vals)
        td = np.zeros((len(pts), 6), np.float32)
        en = np.zeros((len(pts), 6), np.float32)
        sig = np.zeros((len(pts), 36), np.float32)
        b.topo_derivative(pts, td, en, sig)
    for c in range(6):
        _, s_ref = O.bem_interior(pts.astype(np.float64), V, T, u_ref[:, 3 * c:3 * c + 3], vals[:, 3 * c:3 * c + 3],
                                  G0, NU0, disp=False)
        td_ref, en_ref = O.topo_derivative(s_ref, G0, NU0)
        assert rel(sig[:, 6 * c:6 * c + 6], s_ref) < 1e-4, c
        assert rel(td[:, c], td_ref) < 2e-4 and rel(en[:, c], en_ref) < 2e-4, c


def test_eval_td_kind(K):
    """kfmm_eval with the TD kind: D^T and the energy density of the stress sum, per target and
    column, against the oracle's stress sum and Eq. deriv (1e-4 at p = 8)."""
    V, T = W.cube_mesh(4)
    E, nu = 1.0, 0.3
    G = E / (2 * (1 + nu))
    nrm, area, cen = O.tri_geometry(V, T)
    trac = nrm @ np.diag([1.0, 0.0, 0.0]).T
    mask = np.zeros((len(T), 3), np.uint8)
    u, t, info = O.bem_solve_dense(V, T, mask, trac, G, nu, tol=1e-10, restart=100)
    q, w = O.tri_quadrature(V, T)
    qn = np.repeat(nrm, 16, axis=0)
    sl = np.repeat(t, 16, axis=0) * w[:, None]
    dl = -np.repeat(u, 16, axis=0) * w[:, None]
    rng = np.random.default_rng(3)
    pts = rng.uniform(0.2, 0.8, size=(400, 3))
    f32 = lambda a: np.ascontiguousarray(a, np.float32)  # noqa: E731
    qf, nf, slf, dlf, pf = (f32(a) for a in (q, qn, sl, dl, pts))
    # two columns: the solution and twice the solution
    sl2, dl2 = np.concatenate([slf, 2 * slf], axis=1), np.concatenate([dlf, 2 * dlf], axis=1)
    s_ref = O.direct_stress(pf.astype(np.float64), qf.astype(np.float64), nf.astype(np.float64),
                            slf.astype(np.float64), dlf.astype(np.float64), G, nu)
    td_ref, en_ref = O.topo_derivative(s_ref, G, nu)
    with K.Kfmm(p=8, m2l_rtol=1e-7) as f:
        f.set_material(K.material_K(G, nu), G)
        f.build(qf, nf, pf)
        out = np.zeros((len(pts), 4), np.float32)
        f.eval(sl2, dl2, out, K.KFMM_TD, ncol=2)
    assert rel(out[:, 0], td_ref) < 2e-4 and rel(out[:, 1], en_ref) < 2e-4
    assert rel(out[:, 2], 4 * td_ref) < 2e-4 and rel(out[:, 3], 4 * en_ref) < 2e-4
