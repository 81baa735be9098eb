"""Pins of the oracle's collocation BEM (Eq. num, coef, num2), its 16-point rule, its
analytic singular blocks, GMRES and the interior fields, against closed forms, brute-force
integration and dense linear algebra.
"""
import math

import numpy as np
import pytest
from scipy import integrate

import oracle as O
import workloads as W

G0, NU0 = 1.0, 0.3
K0 = 2 * G0 * (1 + NU0) / (3 * (1 - 2 * NU0))


# ----------------------------------------------------------------- 16-point rule
def exact_monomial(V, a, b, c):
    """int over the triangle of l1^a l2^b l3^c = 2 A a! b! c! / (a+b+c+2)!."""
    area = 0.5 * np.linalg.norm(np.cross(V[1] - V[0], V[2] - V[0]))
    return 2 * area * math.factorial(a) * math.factorial(b) * math.factorial(c) / math.factorial(a + b + c + 2)


def test_quadrature_exact_to_degree_3():
    rng = np.random.default_rng(1)
    V = rng.normal(size=(3, 3))
    q, w = O.tri_quadrature(V, np.array([[0, 1, 2]], dtype=np.int32))
    assert q.shape == (16, 3) and w.shape == (16,)
    # barycentric coordinates of the quadrature points
    M = np.stack([V[0] - V[2], V[1] - V[2]], axis=1)
    lam12 = np.linalg.lstsq(M, (q - V[2]).T, rcond=None)[0].T
    lam = np.column_stack([lam12, 1 - lam12.sum(axis=1)])
    assert np.all(lam > 0)  # all points inside
    for a in range(4):
        for b in range(4 - a):
            for c in range(4 - a - b):
                val = np.sum(w * lam[:, 0] ** a * lam[:, 1] ** b * lam[:, 2] ** c)
                assert val == pytest.approx(exact_monomial(V, a, b, c), rel=1e-12, abs=1e-15)
    # the centre sub-triangle's centroid coincides with the collocation point
    assert np.min(np.linalg.norm(q - V.mean(axis=0), axis=1)) < 1e-14


# ----------------------------------------------------------------- singular blocks
TRIS = [np.array([[0.0, 0, 0], [1.0, 0, 0], [0.0, 1.0, 0]]),          # voxel fan triangle
        np.array([[0.1, -0.2, 0.3], [1.3, 0.4, -0.2], [0.2, 0.9, 0.8]]),  # scalene, tilted
        np.array([[0.0, 0, 0], [2.0, 0, 0], [1.9, 0.25, 0.1]])]           # thin


def _polar_sectors(V):
    """Sectors (a, b) of the triangle seen from its centroid, with in-plane frames."""
    xi = V.mean(axis=0)
    n = np.cross(V[1] - V[0], V[2] - V[0])
    n /= np.linalg.norm(n)
    for e in range(3):
        a, b = V[e] - xi, V[(e + 1) % 3] - xi
        t1 = a / np.linalg.norm(a)
        t2 = np.cross(n, t1)
        th_b = math.atan2(b @ t2, b @ t1)
        yield a, b, t1, t2, th_b


def _ray_to_edge(a, b, e):
    """Distance along the in-plane unit direction e from the centroid to the line a-b."""
    # solve rho e = a + s (b - a) in the plane (least squares on 3 equations, exact here)
    M = np.stack([e, -(b - a)], axis=1)
    rho, s = np.linalg.lstsq(M, a, rcond=None)[0]
    return rho


def brute_U_self(V, G, nu):
    """int_tri U(xi - x) dA in polar coordinates about xi: the radial part is exact by
    homogeneity (U(rho e) rho = U(e)), the angle is integrated adaptively in theta with
    the boundary distance R(theta) found by ray-edge intersection."""
    tot = np.zeros((3, 3))
    for a, b, t1, t2, th_b in _polar_sectors(V):
        def f(th):
            e = math.cos(th) * t1 + math.sin(th) * t2
            return O.kernel_U(e, G, nu) * _ray_to_edge(a, b, e)
        val, err = integrate.quad_vec(f, 0.0, th_b, epsabs=1e-13, epsrel=1e-12)
        tot += val * np.sign(th_b)
    return tot


def closed_form_inv_r(V):
    """int_tri dA / |x - xi| = sum_edges h [ln(sec + tan)] between the edge's end angles."""
    tot = 0.0
    for a, b, t1, t2, th_b in _polar_sectors(V):
        d = b - a
        foot = a - (a @ d) / (d @ d) * d           # foot of the perpendicular from xi
        h = np.linalg.norm(foot)
        u = foot / h
        w = d / np.linalg.norm(d)
        ph_a, ph_b = math.atan2(a @ w, a @ u), math.atan2(b @ w, b @ u)
        F = lambda p: math.log(1.0 / math.cos(p) + math.tan(p))
        tot += h * abs(F(ph_b) - F(ph_a))
    return tot


def brute_PV_moment(V):
    """J = PV int (x - xi)/|x - xi|^3 dA = -oint nu / |x - xi| ds (divergence theorem in
    the plane; the small circle around xi contributes int e dtheta = 0)."""
    xi = V.mean(axis=0)
    n = np.cross(V[1] - V[0], V[2] - V[0])
    n /= np.linalg.norm(n)
    J = np.zeros(3)
    for e in range(3):
        a, b = V[e], V[(e + 1) % 3]
        L = np.linalg.norm(b - a)
        nu_out = np.cross(b - a, n) / L
        val, _ = integrate.quad(lambda s: 1.0 / np.linalg.norm(a + s * (b - a) - xi), 0, 1,
                                epsabs=1e-14, epsrel=1e-13)
        J -= nu_out * val * L
    return J, n


@pytest.mark.parametrize("V", TRIS)
@pytest.mark.parametrize("G,nu", [(1.0, 0.3), (2.2, 0.17)])
def test_self_integral_U_brute_force(V, G, nu):
    Us, _ = O.self_integrals(V[0], V[1], V[2], G, nu)
    ref = brute_U_self(V, G, nu)
    assert np.allclose(Us, ref, rtol=1e-9, atol=1e-11 * np.abs(ref).max())
    # trace: (3 (3 - 4nu) + 1) int dA/r / (16 pi G (1 - nu)), with int dA/r in closed form
    tr = (3 * (3 - 4 * nu) + 1) * closed_form_inv_r(V) / (16 * math.pi * G * (1 - nu))
    assert np.trace(Us) == pytest.approx(tr, rel=1e-12)


@pytest.mark.parametrize("V", TRIS)
@pytest.mark.parametrize("nu", [0.3, 0.17])
def test_self_integral_P_principal_value(V, nu):
    """In the element's plane P(xi - x) = A(rhat)/r^2 with A linear in rhat (the kernel is
    pinned separately), so PV int P dA = -(J.t1 A(t1) + J.t2 A(t2)) with J from the
    boundary line integral."""
    _, Ts = O.self_integrals(V[0], V[1], V[2], 1.0, nu)
    J, n = brute_PV_moment(V)
    t1 = (V[1] - V[0]) / np.linalg.norm(V[1] - V[0])
    t2 = np.cross(n, t1)
    ref = -(J @ t1 * O.kernel_T(t1, n, nu) + J @ t2 * O.kernel_T(t2, n, nu))
    assert np.allclose(Ts, ref, rtol=1e-9, atol=1e-12)


def test_self_integral_P_equilateral_vanishes():
    V = np.array([[0.0, 0, 0], [1.0, 0, 0], [0.5, math.sqrt(3) / 2, 0]])
    _, Ts = O.self_integrals(V[0], V[1], V[2], 1.0, 0.3)
    assert np.abs(Ts).max() < 1e-14


# ----------------------------------------------------------------- assembled operators
@pytest.fixture(scope="module")
def sphere2():
    V, T = W.icosphere(2)
    H, Gm = O.bem_assemble(V, T, G0, NU0)
    nrm, area, cen = O.tri_geometry(V, T)
    return V, T, H, Gm, nrm, area, cen


def test_rigid_translation_rows(sphere2):
    """At a smooth collocation point 1/2 I + int P dGamma = 0 (rigid translation)."""
    V, T, H, Gm, nrm, area, cen = sphere2
    nt = len(T)
    rs = H.reshape(nt, 3, nt, 3).sum(axis=2)
    assert np.abs(rs).max() < 2e-3


def test_rigid_rotation_rows(sphere2):
    """u = omega x xi is stress-free: H u = O(h) (piecewise-constant u on each element)."""
    V, T, H, Gm, nrm, area, cen = sphere2
    om = np.array([0.4, -0.9, 0.5])
    u = np.cross(om, cen).reshape(-1)
    r = H @ u
    assert np.abs(r).max() < 0.02 * np.abs(u).max()


def test_single_layer_symmetry_of_blocks(sphere2):
    """U is symmetric and even, so for two far elements U^D_lk ~ U^D_kl^T."""
    V, T, H, Gm, nrm, area, cen = sphere2
    nt = len(T)
    B = Gm.reshape(nt, 3, nt, 3)
    dist = np.linalg.norm(cen - cen[0], axis=1)
    l, k = 0, int(np.argmax(dist))
    assert np.allclose(B[l, :, k, :] / area[k], (B[k, :, l, :] / area[l]).T, rtol=2e-3)


def test_gmres_matches_dense_solve():
    """Mixed BCs (clamped face x = 0, traction on x = 1) on a 2x2x2 voxel cube."""
    V, T = W.cube_mesh(2)
    nrm, area, cen = O.tri_geometry(V, T)
    nt = len(T)
    mask = np.zeros((nt, 3), np.uint8)
    vals = np.zeros((nt, 3))
    mask[cen[:, 0] < 1e-9] = 1
    vals[cen[:, 0] > 1 - 1e-9] = [0.0, 0.0, -1.0]
    H, Gm = O.bem_assemble(V, T, G0, NU0)
    A, b = O.bem_system(H, Gm, mask, vals)
    x, ok, it, rel = O.gmres(A, b, tol=1e-12, restart=60, maxit=2000)
    xd = np.linalg.solve(A, b)
    assert ok and rel <= 1e-12
    assert np.allclose(x, xd, rtol=0, atol=1e-9 * np.abs(xd).max())
    # the rearranged system reproduces H u = Gm t
    u, t = O.unknowns_to_fields(xd, mask, vals)
    assert np.allclose(H @ u.reshape(-1), Gm @ t.reshape(-1), atol=1e-10)


@pytest.mark.parametrize("level", [1, 2])
def test_lame_sphere(level):
    """Solid sphere under t = +n: u_r = r/(3K) after removing the rigid-body modes; the
    error of piecewise-constant collocation is O(h) and halves per refinement."""
    errs = []
    for lev in (level, level + 1):
        V, T = W.icosphere(lev)
        nrm, area, cen = O.tri_geometry(V, T)
        mask = np.zeros((len(T), 3), np.uint8)
        u, t, info = O.bem_solve_dense(V, T, mask, nrm, G0, NU0, tol=1e-10, restart=60)
        assert info["converged"]
        u = O.remove_rigid_modes(u, cen, area)
        rr = np.linalg.norm(cen, axis=1)
        ur = np.einsum("ij,ij->i", u, cen / rr[:, None])
        errs.append(np.abs(ur / (rr / (3 * K0)) - 1).max())
    assert errs[0] < 0.06 and errs[1] < 0.6 * errs[0]


def test_lame_shell():
    """Thick shell a=0.5, b=1 with inner pressure p: u_r = p a^3/(b^3-a^3) [r/(3K) + b^3/(4G r^2)]."""
    a, b, p = 0.5, 1.0, 1.0
    Vo, To = W.icosphere(2, radius=b)
    Vi, Ti = W.icosphere(2, radius=a, inward=True)  # normal out of the material = into the hole
    V = np.vstack([Vo, Vi])
    T = np.vstack([To, Ti + len(Vo)]).astype(np.int32)
    nrm, area, cen = O.tri_geometry(V, T)
    nt_o = len(To)
    trac = np.zeros((len(T), 3))
    trac[nt_o:] = -p * nrm[nt_o:]  # pressure pushes on the material: t = -p n
    mask = np.zeros((len(T), 3), np.uint8)
    u, t, info = O.bem_solve_dense(V, T, mask, trac, G0, NU0, tol=1e-10, restart=100)
    assert info["converged"]
    u = O.remove_rigid_modes(u, cen, area)
    rr = np.linalg.norm(cen, axis=1)
    ur = np.einsum("ij,ij->i", u, cen / rr[:, None])
    ex = p * a ** 3 / (b ** 3 - a ** 3) * (rr / (3 * K0) + b ** 3 / (4 * G0 * rr ** 2))
    assert np.abs(ur / ex - 1).max() < 0.08


def _gl_triangle_block(A, B, C, x, n, G, nu, m=48):
    """int_T U and int_T T(., n) at x by a tensor Gauss-Legendre rule on the collapsed square
    (y = A + u (B - A) + (1 - u) w (C - A), dA = 2 |T| (1 - u) du dw): independent of the
    midpoint-subdivision rule it checks."""
    g, wg = np.polynomial.legendre.leggauss(m)
    g, wg = 0.5 * (g + 1), 0.5 * wg
    area = 0.5 * np.linalg.norm(np.cross(B - A, C - A))
    U, T = np.zeros((3, 3)), np.zeros((3, 3))
    for u, wu in zip(g, wg):
        for w_, ww in zip(g, wg):
            y = A + u * (B - A) + (1 - u) * w_ * (C - A)
            wt = 2 * area * (1 - u) * wu * ww
            U += wt * O.kernel_U(x - y, G, nu)
            T += wt * O.kernel_T(x - y, n, nu)
    return U, T


def test_upsampled_near_block_converges():
    """The upsampled quadrature of a triangle next to the collocation point (Sec. "Matrix-
    vector products"): the 4-node rule on 4^s sub-triangles converges to the integral (an
    independent tensor Gauss-Legendre rule), its error falling ~16x per level (degree-3 rule,
    h^4), from ~1e-3 at the 16-point rule to < 1e-6 at 4^4 sub-triangles."""
    G, nu = 1.3, 0.27
    V, T = W.icosphere(2)
    nrm, area, cen = O.tri_geometry(V, T)
    k = next(i for i in range(1, len(T)) if len(set(T[i]) & set(T[0])) == 1)  # shares one vertex
    ref_U, ref_T = _gl_triangle_block(*V[T[k]], cen[0], nrm[k], G, nu)
    errs = []
    for lev in range(1, 5):
        Ub, Tb = O.tri_block(*V[T[k]], cen[0], levels=lev, G=G, nu=nu)
        errs.append(max(np.abs(Ub - ref_U).max() / np.abs(ref_U).max(), np.abs(Tb - ref_T).max() / np.abs(ref_T).max()))
    assert errs[0] > 1e-5 and errs[-1] < 1e-6, errs
    assert all(b < a / 8 for a, b in zip(errs, errs[1:])), errs
    # levels = 1 is the 16-point rule of the dense operator
    H, Gm = O.bem_assemble(V, T, G, nu)
    Ub, Tb = O.tri_block(*V[T[k]], cen[0], levels=1, G=G, nu=nu)
    assert np.allclose(Gm[0:3, 3 * k:3 * k + 3], Ub, rtol=0, atol=1e-13 * np.abs(Ub).max())
    assert np.allclose(H[0:3, 3 * k:3 * k + 3], Tb, rtol=0, atol=1e-13 * np.abs(Tb).max())


def test_upsampled_near_blocks_restore_rigid_translation():
    """A rigid translation solves the homogeneous problem: 1/2 u + P u = 0 on a closed surface.
    The discrete rows of H fail that by the quadrature error, dominated by the triangles next
    to the collocation point; upsampling them (4^3 sub-triangles) cuts the worst row >= 20x,
    and leaves the blocks of the other triangles unchanged."""
    V, T = W.icosphere(2)
    errs = []
    for lev in (1, 3):
        H, Gm = O.bem_assemble(V, T, G0, NU0, near_levels=lev)
        tr = np.zeros((len(T), 3))
        tr[:, 0] = 1.0
        errs.append(np.abs(H @ tr.reshape(-1)).max())
        if lev == 1:
            H1 = H
    assert errs[1] < errs[0] / 20, errs
    near = np.zeros((len(T), len(T)), bool)
    for l in range(len(T)):
        for k in range(len(T)):
            near[l, k] = k != l and len(set(T[l]) & set(T[k])) > 0
    far = np.repeat(np.repeat(~near, 3, axis=0), 3, axis=1)
    assert np.array_equal(H[far], H1[far])


def test_spherical_cavity_exterior_problem():
    """Exterior problem (the void surfaces of a periodic cell, Sec. "Periodic cell of a
    metamaterial"): a spherical cavity of radius a in an infinite medium, normals out of the
    material (into the cavity), internal pressure p, i.e. t = p e_r on the cavity wall.  The
    closed form is u_r = p a^3 / (4 G r^2): p a / (4 G) on the wall, which the element values
    approach at O(h) (the error halves per refinement: 3.9% and 1.9% at 320 and 1280
    triangles), and within 1% in the material (r = 2a, 3a, 2.1a, through the representation
    formula).  No rigid mode: the exterior traction problem is uniquely solvable.  Also the
    hydrostatic unit-strain load case: t = -sigma^h n with sigma^h = 3K I gives the same
    field with p = 3K."""
    a, p, G, nu = 0.4, 1.0, 1.3, 0.27
    Kb = 2 * G * (1 + nu) / (3 * (1 - 2 * nu))
    errs = []
    for lev in (2, 3):
        V, T = W.icosphere(lev, radius=a, inward=True)
        nrm, area, cen = O.tri_geometry(V, T)
        rr = np.linalg.norm(cen, axis=1)
        er = cen / rr[:, None]
        mask = np.zeros((len(T), 3), np.uint8)
        cols = [p * er, -(3 * Kb) * nrm]  # internal pressure; hydrostatic macro strain (S = 3K)
        for k, trac in enumerate(cols):
            u, t, info = O.bem_solve_dense(V, T, mask, trac, G, nu, tol=1e-11, restart=100)
            assert info["converged"]
            pk = p if k == 0 else 3 * Kb
            ur = np.einsum("ij,ij->i", u, er)
            err = np.abs(ur / (pk * a / (4 * G)) - 1).max()
            # tangential displacement vanishes by symmetry
            assert np.linalg.norm(u - ur[:, None] * er) / np.linalg.norm(u) < 2 * err + 1e-3
            if k == 0:
                errs.append(err)
                pts = np.array([[2 * a, 0, 0], [0, -3 * a, 0], [1.2 * a, 1.2 * a, 1.2 * a]])
                dsp, _ = O.bem_interior(pts, V, T, u, t, G, nu, stress=False)
                rp = np.linalg.norm(pts, axis=1)
                urp = np.einsum("ij,ij->i", dsp, pts / rp[:, None])
                assert np.abs(urp / (p * a ** 3 / (4 * G * rp ** 2)) - 1).max() < 0.01
    assert errs[0] < 0.05 and errs[1] < 0.6 * errs[0], errs


def test_uniform_tension_cube_interior():
    """Sec. "Performance and scalability" benchmark: unit cube, E = 1, nu = 0.3, uniform
    tension s = 1 along x.  The interior stress is s e1 e1 and D^T = 1.00227."""
    E, nu = 1.0, 0.3
    G = E / (2 * (1 + nu))
    V, T = W.cube_mesh(3)
    nrm, area, cen = O.tri_geometry(V, T)
    sig = np.diag([1.0, 0.0, 0.0])
    trac = nrm @ sig.T
    mask = np.zeros((len(T), 3), np.uint8)
    u, t, info = O.bem_solve_dense(V, T, mask, trac, G, nu, tol=1e-10, restart=100)
    assert info["converged"]
    pts = np.array([[0.5, 0.5, 0.5], [0.4, 0.6, 0.45]])
    dsp, st = O.bem_interior(pts, V, T, u, t, G, nu)
    assert np.allclose(st[:, 0], 1.0, atol=0.03)
    assert np.abs(st[:, 1:]).max() < 0.03
    td, en = O.topo_derivative(st, G, nu)
    assert td == pytest.approx(np.full(2, 1.0022727272727273), rel=0.06)
    # strain gradient of the recovered displacement: du_x/dx = s/E
    d2, _ = O.bem_interior(np.array([[0.4, 0.5, 0.5], [0.6, 0.5, 0.5]]), V, T, u, t, G, nu, stress=False)
    assert (d2[1, 0] - d2[0, 0]) / 0.2 == pytest.approx(1.0 / E, rel=0.05)


# ----------------------------------------------------------------- mesh generator counts
def test_voxel_mesh_dof_counts():
    """24 N^2 triangles; N = 64 gives the 4.72e6 source DOFs (3*16 per triangle) and the
    0.79e6 volume DOFs (3 N^3) quoted for the cantilever example."""
    for n in (1, 2, 5):
        V, T = W.cube_mesh(n)
        assert len(T) == 24 * n * n
    n = 64
    V, T = W.cube_mesh(n)
    assert len(T) == 98304
    assert 3 * 16 * len(T) == 4718592
    assert 3 * n ** 3 == 786432
    nrm, area, cen = O.tri_geometry(V, T)
    assert area.sum() == pytest.approx(6.0, rel=1e-12)
    # outward normals: centroid moves outward along n
    assert np.all(np.einsum("ij,ij->i", nrm, cen - 0.5) > 0)
