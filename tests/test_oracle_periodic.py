"""Pins of the oracle's periodic sums (Sec. "Periodic cell of a metamaterial": the sums over
the infinite periodic surface of a cubic cell) against facts fixed by elasticity and by
lattice sums, not by the oracle itself.

The periodic single layer is the Fourier series of Eq. disp_1 without k = 0, the double layer
its traction kernel; the oracle sums both by Ewald's split.  A slip in either half of the split
(a wrong screening function, a dropped factor (1 + k^2/4 xi^2), a wrong mean term) breaks
the independence of the screening parameter; a wrong normalisation or Poisson-ratio coupling
breaks the Navier equation; a wrong constant breaks the cubic-lattice constant; a wrong sign,
Lame constant or index in the double layer breaks the rigid-translation identity.
"""
import numpy as np

import oracle as O

G, NU = 1.3, 0.3
LAM = 2 * G * NU / (1 - 2 * NU)
RNG = np.random.default_rng(21)


def sphere_quadrature(y0, R, nt=24, nph=48):
    """Gauss-Legendre in cos(theta) x trapezoid in phi on a sphere: points, outward normals,
    weights (spectrally accurate for integrands smooth on the sphere)."""
    xg, wg = np.polynomial.legendre.leggauss(nt)
    th, ph = np.arccos(xg), 2 * np.pi * np.arange(nph) / nph
    T, P = np.meshgrid(th, ph, indexing="ij")
    n = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    w = np.repeat(wg, nph) * (2 * np.pi / nph) * R * R
    return y0 + R * n, n, w


def test_regular_part_is_the_cubic_lattice_constant():
    """lim_{d->0} [U_per(d) - U(d)] for the simple cubic lattice.  At nu = 1/2 Eq. disp_1 is the
    Stokeslet / (8 pi G) and the limit is Hasimoto's -2.837297 / (6 pi G Lc) I (the leading
    wall-interaction term of the drag on a cubic array of spheres, Hasimoto 1959).  For any nu the
    Laplace part carries the same lattice constant, -2.837297 / (4 pi Lc), and the d_i d_j psi part
    a third of it by cubic symmetry: (1 - 1 / (6 (1 - nu))) -2.837297 / (4 pi G Lc) I."""
    zeta = 2.8372974794806
    for Lc in (1.0, 2.5):
        U, dU = O.periodic_U(np.zeros(3), G=G, nu=0.5 - 1e-13, Lc=Lc)
        np.testing.assert_allclose(U, -zeta / (6 * np.pi * G * Lc) * np.eye(3), rtol=1e-9, atol=1e-14)
        assert np.abs(dU).max() < 1e-12
        U, _ = O.periodic_U(np.zeros(3), G=G, nu=NU, Lc=Lc)
        pred = -zeta / (4 * np.pi * G * Lc) * (1 - 1 / (6 * (1 - NU)))
        np.testing.assert_allclose(U, pred * np.eye(3), rtol=1e-9, atol=1e-14)


def test_independent_of_the_ewald_parameter():
    """The split moves weight between the real and reciprocal sums; their total is fixed."""
    for _ in range(4):
        d = RNG.uniform(-0.6, 0.6, 3)
        ref = O.periodic_U(d, G, NU, 1.0, xi=2.0)
        for xi in (4.5, 9.0):
            U, dU = O.periodic_U(d, G, NU, 1.0, xi=xi)
            np.testing.assert_allclose(U, ref[0], rtol=1e-11, atol=1e-13)
            np.testing.assert_allclose(dU, ref[1], rtol=1e-10, atol=1e-12)
    src = RNG.uniform(0, 1, (40, 3))
    nrm = RNG.normal(size=(40, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    sl, dl = RNG.normal(size=(40, 3)), RNG.normal(size=(40, 3))
    trg = RNG.uniform(0, 1, (7, 3))
    a = O.periodic_disp(trg, src, nrm, sl, dl, G, NU, 1.0, xi=3.0)
    b = O.periodic_disp(trg, src, nrm, sl, dl, G, NU, 1.0, xi=7.0)
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12 * np.abs(a).max())


def test_periodic_in_every_direction():
    d = np.array([0.21, -0.33, 0.08])
    U0, dU0 = O.periodic_U(d, G, NU, 1.7)
    for a in range(3):
        for s in (-1, 2):
            e = np.zeros(3)
            e[a] = s * 1.7
            U, dU = O.periodic_U(d + e, G, NU, 1.7)
            np.testing.assert_allclose(U, U0, rtol=1e-11, atol=1e-13)
            np.testing.assert_allclose(dU, dU0, rtol=1e-10, atol=1e-12)


def test_navier_equation_with_the_balancing_body_force():
    """u = U_per F solves G lap u + (lambda + G) grad div u = -F delta + F / V: away from the
    force the operator returns the uniform body force F / V that the missing k = 0 term adds."""
    F = np.array([0.3, -1.0, 0.7])
    for Lc, x in ((1.0, np.array([0.31, 0.22, -0.17])), (2.0, np.array([-0.5, 0.7, 0.4]))):
        def u(p):
            return O.periodic_U(p, G, NU, Lc)[0] @ F

        h = 2e-3 * Lc
        H = np.zeros((3, 3, 3))  # d2 u_c / dx_a dx_b, fourth-order differences
        for a in range(3):
            for b in range(3):
                ea, eb = np.eye(3)[a] * h, np.eye(3)[b] * h

                def d2(s):
                    return (u(x + s * ea + s * eb) - u(x + s * ea - s * eb) - u(x - s * ea + s * eb)
                            + u(x - s * ea - s * eb)) / (4 * s * s * h * h)

                H[:, a, b] = (4 * d2(1.0) - d2(2.0)) / 3
        nav = G * np.einsum("caa->c", H) + (LAM + G) * np.einsum("aac->c", H)
        np.testing.assert_allclose(nav, F / Lc ** 3, rtol=2e-4, atol=2e-4 * np.abs(F).max() / Lc ** 3)


def test_free_space_double_layer_is_the_traction_of_the_single_layer():
    """The double layer is built as -[lambda n_j dU_mi/dd_m + G n_k (dU_ki/dd_j + dU_ji/dd_k)];
    with the free-space U this reproduces Eq. disp_2 exactly."""
    for _ in range(3):
        d, n = RNG.normal(size=3), RNG.normal(size=3)
        n /= np.linalg.norm(n)
        h = 1e-5
        dU = np.zeros((3, 3, 3))
        for m in range(3):
            e = np.eye(3)[m] * h
            dU[:, :, m] = (-O.kernel_U(d + 2 * e, G, NU) + 8 * O.kernel_U(d + e, G, NU)
                           - 8 * O.kernel_U(d - e, G, NU) + O.kernel_U(d - 2 * e, G, NU)) / (12 * h)
        T = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                div = sum(dU[m, i, m] for m in range(3))
                T[i, j] = -(LAM * n[j] * div + G * sum(n[k] * (dU[k, i, j] + dU[j, i, k]) for k in range(3)))
        np.testing.assert_allclose(T, O.kernel_T(d, n, NU), rtol=1e-8, atol=1e-10)


def test_double_layer_of_a_rigid_translation():
    """For a closed surface S bounding B (outward normals), the divergence theorem with the
    periodic field (div sigma = -delta + 1/V) gives int_S T_per c dS = c (|B|/V - chi_B(x)):
    -c (1 - |B|/V) inside B, c |B|/V outside, for any cell size and Poisson ratio."""
    for Lc, nu in ((1.0, NU), (1.6, 0.1)):
        R, y0 = 0.22 * Lc, np.array([0.05, -0.1, 0.12]) * Lc
        src, nrm, w = sphere_quadrature(y0, R)
        c = np.array([0.4, 1.0, -0.6])
        trg = y0 + np.array([[0.03, 0.02, -0.05], [0.4, 0.1, 0.2], [-0.45, 0.3, 0.05]]) * Lc
        out = O.periodic_disp(trg, src, nrm, None, w[:, None] * c[None, :], G, nu, Lc)
        f = 4 / 3 * np.pi * R ** 3 / Lc ** 3
        np.testing.assert_allclose(out[0], c * (f - 1), rtol=1e-9)
        np.testing.assert_allclose(out[1:], np.tile(c * f, (2, 1)), rtol=1e-8)


def test_single_layer_of_a_uniform_stress_traction():
    """t = sigma n on a sphere (sigma constant) has no net force; the periodic single layer of it
    is the field of the cavity's equivalent force dipole and, by the same divergence argument
    with the reciprocal identity, int_S U_per (sigma n) dS = -int_B grad(U_per) : sigma dV; at a
    point outside B with a small sphere this is the dipole field -dU_per/dd_k sigma_jk |B|
    to O(R^2) relative."""
    sig = np.array([[1.0, 0.3, -0.2], [0.3, -0.5, 0.4], [-0.2, 0.4, 0.8]])
    R, y0 = 0.01, np.array([0.2, 0.1, -0.15])
    src, nrm, w = sphere_quadrature(y0, R, 12, 24)
    x = np.array([0.55, -0.2, 0.3])
    out = O.periodic_disp(x[None, :], src, nrm, w[:, None] * (nrm @ sig.T), None, G, NU, 1.0)[0]
    _, dU = O.periodic_U(x - y0, G, NU, 1.0)
    pred = -np.einsum("ijk,jk->i", dU, sig) * (4 / 3 * np.pi * R ** 3)
    np.testing.assert_allclose(out, pred, rtol=2e-3)


def test_batched_sum_matches_the_kernel_pair_by_pair():
    """The structure-factor form of the reciprocal sum equals the sum of the periodic kernel over
    the pairs (a reordering of the same finite sum)."""
    src = RNG.uniform(0, 1, (12, 3))
    nrm = RNG.normal(size=(12, 3))
    nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
    sl, dl = RNG.normal(size=(12, 3)), RNG.normal(size=(12, 3))
    trg = np.vstack([RNG.uniform(0, 1, (3, 3)), src[:2]])  # two targets on sources
    got = O.periodic_disp(trg, src, nrm, sl, dl, G, NU, 1.0)
    ref = np.zeros_like(got)
    for i, x in enumerate(trg):
        for j in range(len(src)):
            U, dU = O.periodic_U(x - src[j], G, NU, 1.0)
            n = nrm[j]
            T = np.zeros((3, 3))
            for p in range(3):
                for q in range(3):
                    div = sum(dU[m, p, m] for m in range(3))
                    T[p, q] = -(LAM * n[q] * div + G * sum(n[m] * (dU[m, p, q] + dU[q, p, m]) for m in range(3)))
            ref[i] += U @ sl[j] + T @ dl[j]
    np.testing.assert_allclose(got, ref, rtol=1e-10, atol=1e-12 * np.abs(ref).max())
