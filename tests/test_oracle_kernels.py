"""Pins of the oracle's four kernels (Eq. disp_1, disp_2, stress_2, stress_3) and of the
topological derivative (Eq. deriv) against facts fixed by elasticity, not by the oracle.

Every pin is chosen so a plausible slip (a constant off by 4 as printed in Eq. stress_2, a
missing G in Eq. stress_3, a sign or an index swap in the antisymmetric term of
Eq. disp_2) fails at least one of them.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W

VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]


def hooke(eps, G, nu):
    """Eq. elast: C_ijkl = K d_ij d_kl + G (d_ik d_jl + d_il d_jk - 2/3 d_ij d_kl)."""
    K = 2.0 * G * (1.0 + nu) / (3.0 * (1.0 - 2.0 * nu))
    tr = np.trace(eps)
    return K * tr * np.eye(3) + 2.0 * G * (eps - tr / 3.0 * np.eye(3))


def voigt(s):
    return np.array([s[i, j] for i, j in VOIGT])


def fd_grad(field, p, h=1e-5):
    """grad[a, b] = d field_a / d p_b by 4th-order central differences."""
    g = np.zeros((3, 3))
    for b in range(3):
        e = np.zeros(3)
        e[b] = h
        g[:, b] = (-field(p + 2 * e) + 8 * field(p + e) - 8 * field(p - e) + field(p - 2 * e)) / (12 * h)
    return g


RNG = np.random.default_rng(11)
POINTS = [RNG.normal(size=3) for _ in range(4)]
NORMALS = [v / np.linalg.norm(v) for v in (RNG.normal(size=3) for _ in range(4))]
MATERIALS = [(1.0, 0.3), (2.7, 0.21), (0.45, 0.37)]


@pytest.mark.parametrize("G,nu", MATERIALS)
def test_U_symmetry_and_homogeneity(G, nu):
    for d in POINTS:
        U = O.kernel_U(d, G, nu)
        assert np.allclose(U, U.T, rtol=0, atol=1e-15)
        assert np.allclose(O.kernel_U(-d, G, nu), U, rtol=1e-14)
        assert np.allclose(O.kernel_U(2.5 * d, G, nu), U / 2.5, rtol=1e-13)
        for n in NORMALS:
            assert np.allclose(O.kernel_T(3.0 * d, n, nu), O.kernel_T(d, n, nu) / 9.0, rtol=1e-13)
    assert np.all(O.kernel_U(np.zeros(3), G, nu) == 0)
    assert np.all(O.kernel_T(np.zeros(3), NORMALS[0], nu) == 0)
    assert np.all(O.kernel_D(np.zeros(3), nu) == 0)
    assert np.all(O.kernel_S(np.zeros(3), NORMALS[0], G, nu) == 0)


@pytest.mark.parametrize("G,nu", MATERIALS)
def test_U_solves_navier(G, nu):
    """div sigma(U e_k) = 0 away from the point force (Eq. elast with no body force)."""
    for k in range(3):
        def sig(p):
            eps_field = lambda q: O.kernel_U(q, G, nu)[:, k]
            gr = fd_grad(eps_field, p, 1e-4)
            return hooke(0.5 * (gr + gr.T), G, nu)
        for p in POINTS[:2]:
            div = np.zeros(3)
            for j in range(3):
                div += fd_grad(lambda q: sig(q)[:, j], p, 2e-3)[:, j]
            scale = np.abs(sig(p)).max() / np.linalg.norm(p)
            assert np.abs(div).max() < 1e-7 * scale


def sphere_rule(nth=24, nph=48):
    x, w = np.polynomial.legendre.leggauss(nth)
    ph = np.arange(nph) * 2 * np.pi / nph
    ct, phi = np.meshgrid(x, ph, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    n = np.stack([st * np.cos(phi), st * np.sin(phi), ct], axis=-1).reshape(-1, 3)
    wt = (np.repeat(w, nph) * 2 * np.pi / nph)
    return n, wt


@pytest.mark.parametrize("G,nu", MATERIALS)
def test_D_point_force_equilibrium(G, nu):
    """A sphere around a unit point force e_k carries total traction -e_k: the printed
    1/(2 pi) constant of Eq. stress_2 would give -4 e_k."""
    n, wt = sphere_rule()
    R = 0.7
    for k in range(3):
        tot = np.zeros(3)
        for nn, ww in zip(n, wt):
            Dk = O.kernel_D(R * nn, nu)[k]
            s = np.zeros((3, 3))
            for c, (i, j) in enumerate(VOIGT):
                s[i, j] = s[j, i] = Dk[c]
            tot += s @ nn * ww * R * R
        assert np.allclose(tot, -np.eye(3)[k], atol=1e-12)


@pytest.mark.parametrize("G,nu", MATERIALS)
def test_D_is_hooke_of_grad_U(G, nu):
    for d in POINTS:
        Dm = O.kernel_D(d, nu)
        for k in range(3):
            gr = fd_grad(lambda q: O.kernel_U(q, G, nu)[:, k], d)
            ref = voigt(hooke(0.5 * (gr + gr.T), G, nu))
            assert np.allclose(Dm[k], ref, rtol=1e-8, atol=1e-9 * np.abs(ref).max())


@pytest.mark.parametrize("G,nu", MATERIALS)
def test_T_is_traction_of_point_force(G, nu):
    """T_ij(xi - x, n) = traction_j at x (normal n) of the point force e_i at xi, i.e.
    -sum_l D_i,jl(xi - x) n_l.  Pins the sign and index order of the antisymmetric term."""
    for d in POINTS:
        Dm = O.kernel_D(d, nu)
        for n in NORMALS:
            Tm = O.kernel_T(d, n, nu)
            for i in range(3):
                s = np.zeros((3, 3))
                for c, (a, b) in enumerate(VOIGT):
                    s[a, b] = s[b, a] = Dm[i, c]
                assert np.allclose(Tm[i], -s @ n, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("G,nu", MATERIALS)
def test_S_is_hooke_of_grad_T(G, nu):
    """Eq. stress_3 with the factor G: the stress of the double-layer field."""
    for d in POINTS:
        for n in NORMALS[:2]:
            Sm = O.kernel_S(d, n, G, nu)
            for k in range(3):
                gr = fd_grad(lambda q: O.kernel_T(q, n, nu)[:, k], d)
                ref = voigt(hooke(0.5 * (gr + gr.T), G, nu))
                assert np.allclose(Sm[k], ref, rtol=1e-7, atol=1e-8 * np.abs(ref).max())


# ----------------------------------------------------------------- surface identities
@pytest.fixture(scope="module")
def sphere_quad():
    V, T = W.icosphere(3, radius=1.3, center=(0.2, -0.1, 0.3))
    q, w = O.tri_quadrature(V, T)
    nrm, _, _ = O.tri_geometry(V, T)
    return q, w, np.repeat(nrm, 16, axis=0), np.array([0.2, -0.1, 0.3])


def test_double_layer_rigid_translation(sphere_quad):
    """int_Gamma P e dGamma = -e inside, 0 outside a closed surface."""
    q, w, qn, c = sphere_quad
    pts = np.array([c + [0.1, 0.2, -0.3], c + [0.0, 0.0, 0.0], c + [3.0, 0.0, 0.0]])
    for e in np.eye(3):
        out = O.direct_disp(pts, q, qn, None, np.tile(e, (len(q), 1)) * w[:, None], nu=0.27)
        assert np.allclose(out[:2], -e, atol=2e-6)
        assert np.allclose(out[2], 0, atol=1e-9)


def test_double_layer_rigid_rotation(sphere_quad):
    """u = omega x y is stress-free, so u(p) + int P u = 0 inside: pins the
    antisymmetric (1-2nu)(r_i n_j - r_j n_i) term of Eq. disp_2."""
    q, w, qn, c = sphere_quad
    om = np.array([0.3, -1.1, 0.7])
    u = np.cross(om, q)
    pts = c + np.array([[0.1, 0.2, -0.3], [-0.4, 0.1, 0.2]])
    out = O.direct_disp(pts, q, qn, None, u * w[:, None], nu=0.27)
    assert np.allclose(out, -np.cross(om, pts), atol=5e-6)


@pytest.mark.parametrize("G,nu", [(1.0, 0.3), (2.7, 0.21)])
def test_patch_displacement_and_stress(sphere_quad, G, nu):
    """Linear field u = eps y, t = C:eps n on a closed surface: the interior representation
    u(p) = int U t - int P u returns eps p and Eq. stress_1 returns C:eps (G != 1 pins
    the factor G of Eq. stress_3)."""
    q, w, qn, c = sphere_quad
    rng = np.random.default_rng(5)
    a = rng.normal(size=(3, 3))
    eps = 0.5 * (a + a.T)
    sig = hooke(eps, G, nu)
    u = q @ eps.T
    t = qn @ sig.T
    pts = c + np.array([[0.1, 0.2, -0.3], [-0.4, 0.1, 0.2], [0.0, 0.0, 0.0]])
    dsp = O.direct_disp(pts, q, qn, t * w[:, None], -u * w[:, None], G, nu)
    assert np.allclose(dsp, pts @ eps.T, atol=2e-5)
    st = O.direct_stress(pts, q, qn, t * w[:, None], -u * w[:, None], G, nu)
    assert np.allclose(st, np.tile(voigt(sig), (3, 1)), atol=5e-5 * np.abs(sig).max())


def test_sphere_centre_split(sphere_quad):
    """Hydrostatic traction s n with u = s y/(3K) on a sphere: at the centre the single
    layer gives s(1+nu)/(3(1-nu)) and the double layer s(2-4nu)/(3(1-nu)) (they sum to s)."""
    q, w, qn, c = sphere_quad
    G, nu, s = 1.7, 0.3, 1.0
    K = 2 * G * (1 + nu) / (3 * (1 - 2 * nu))
    # use the exact sphere normal/radius at the quadrature points (flat-facet error aside)
    rad = q - c
    nn = rad / np.linalg.norm(rad, axis=1, keepdims=True)
    sl = s * nn * w[:, None]
    dl = -s * rad / (3 * K) * w[:, None]
    p = c[None, :]
    s_sl = O.direct_stress(p, q, nn, sl, None, G, nu)[0]
    s_dl = O.direct_stress(p, q, nn, None, dl, G, nu)[0]
    assert np.allclose(s_sl[:3], s * (1 + nu) / (3 * (1 - nu)), rtol=2e-3)
    assert np.allclose(s_dl[:3], s * (2 - 4 * nu) / (3 * (1 - nu)), rtol=2e-3)
    assert np.allclose(s_sl[3:], 0, atol=1e-6) and np.allclose(s_dl[3:], 0, atol=1e-6)


# ----------------------------------------------------------------- Eq. deriv
def test_topological_derivative_closed_forms():
    G, nu = 1.0, 0.3
    E = 2 * G * (1 + nu)
    hyd = np.array([[1.0, 1.0, 1.0, 0, 0, 0]])
    td, en = O.topo_derivative(hyd, G, nu)
    assert td[0] == pytest.approx(9 * (1 - nu) / (4 * E), rel=1e-14)
    assert td[0] == pytest.approx(0.6057692307692307, rel=1e-12)
    # uniaxial tension s=1 at E = 1, nu = 0.3
    Gu = 1.0 / (2 * 1.3)
    td, en = O.topo_derivative(np.array([[1.0, 0, 0, 0, 0, 0]]), Gu, 0.3)
    assert td[0] == pytest.approx(3 * 0.7 * (9 + 1.5) / (4 * 1.0 * (7 - 1.5)), rel=1e-13)
    assert td[0] == pytest.approx(1.0022727272727273, rel=1e-12)
    assert en[0] == pytest.approx(0.5, rel=1e-13)  # 1/2 s^2 / E
    # non-negativity: D^T = c [10(1+nu)|dev s|^2 + (7-5nu)/3 tr^2]
    rng = np.random.default_rng(3)
    s = rng.normal(size=(200, 6))
    td, en = O.topo_derivative(s, G, nu)
    S = np.zeros((200, 3, 3))
    for c_, (i, j) in enumerate(VOIGT):
        S[:, i, j] = S[:, j, i] = s[:, c_]
    tr = np.trace(S, axis1=1, axis2=2)
    dev = S - tr[:, None, None] / 3 * np.eye(3)
    alt = 3 * (1 - nu) / (4 * E * (7 - 5 * nu)) * (10 * (1 + nu) * np.einsum("nij,nij->n", dev, dev)
                                                  + (7 - 5 * nu) / 3 * tr ** 2)
    assert np.allclose(td, alt, rtol=1e-12)
    assert np.all(td >= 0) and np.all(en >= 0)
