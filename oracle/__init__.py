"""FP64 CPU oracle for the Kelvin elasticity sums and collocation BEM (arXiv 1612.04082).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` use it; the product package never imports it.  The arithmetic lives in
``kelvin_oracle.c`` (plain C, FP64, OpenMP over targets); this module only compiles it with
gcc and marshals numpy arrays.  It shares no code with the CUDA path.

Paper references (sections / equations of the paper):
  kernel_U  -- Eq. disp_1          kernel_T -- Eq. disp_2
  kernel_D  -- Eq. stress_2        kernel_S -- Eq. stress_3 (with the factor G)
  direct_disp / direct_stress     -- Eq. fmm_summation, summed over all pairs
  tri_quadrature                  -- Sec. "Matrix-vector products" (16-point rule)
  self_integrals, bem_assemble    -- Eq. num, Eq. coef (singular blocks analytic)
  bem_system                      -- Eq. num2
  gmres                           -- Sec. "Discretization of BIE" (GMRES)
  bem_interior                    -- Eq. stress_1 and the BIE at interior points
  topo_derivative                 -- Eq. deriv and the integrand of Eq. functional
  periodic_U, periodic_disp       -- Sec. "Periodic cell of a metamaterial": the sums over the
                                     periodic surface (Fourier series of Eq. disp_1 without
                                     k = 0, by Ewald's split)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kelvin_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "libkelvin_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, OpenMP, no fast-math)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
    return _lib


_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def kernel_U(d, G, nu):
    d = _f64(d).reshape(3)
    out = np.zeros(9)
    _load().ko_kernel_U(_dp(d), ctypes.c_double(G), ctypes.c_double(nu), _dp(out))
    return out.reshape(3, 3)


def kernel_T(d, n, nu):
    d, n = _f64(d).reshape(3), _f64(n).reshape(3)
    out = np.zeros(9)
    _load().ko_kernel_T(_dp(d), _dp(n), ctypes.c_double(nu), _dp(out))
    return out.reshape(3, 3)


def kernel_D(d, nu):
    """[k, s]: stress component s (xx,yy,zz,yz,xz,xy) from SL component k."""
    d = _f64(d).reshape(3)
    out = np.zeros(18)
    _load().ko_kernel_D(_dp(d), ctypes.c_double(nu), _dp(out))
    return out.reshape(3, 6)


def kernel_S(d, n, G, nu):
    d, n = _f64(d).reshape(3), _f64(n).reshape(3)
    out = np.zeros(18)
    _load().ko_kernel_S(_dp(d), _dp(n), ctypes.c_double(G), ctypes.c_double(nu), _dp(out))
    return out.reshape(3, 6)


def direct_disp(trg, src, nrm=None, sl=None, dl=None, G=1.0, nu=0.3):
    """out[i] = sum_j U(x_i - y_j) sl_j + T(x_i - y_j, n_j) dl_j, r = 0 skipped."""
    trg, src, nrm, sl, dl = (_f64(a) for a in (trg, src, nrm, sl, dl))
    if dl is not None and nrm is None:
        raise ValueError("double-layer density needs normals")
    out = np.zeros((trg.shape[0], 3))
    _load().ko_direct_disp(_dp(trg), ctypes.c_int64(trg.shape[0]), _dp(src), _dp(nrm), _dp(sl),
                           _dp(dl), ctypes.c_int64(src.shape[0]), ctypes.c_double(G),
                           ctypes.c_double(nu), _dp(out))
    return out


def direct_stress(trg, src, nrm=None, sl=None, dl=None, G=1.0, nu=0.3):
    """out[i] = sum_j D(x_i - y_j) sl_j + S(x_i - y_j, n_j) dl_j, Voigt xx,yy,zz,yz,xz,xy."""
    trg, src, nrm, sl, dl = (_f64(a) for a in (trg, src, nrm, sl, dl))
    if dl is not None and nrm is None:
        raise ValueError("double-layer density needs normals")
    out = np.zeros((trg.shape[0], 6))
    _load().ko_direct_stress(_dp(trg), ctypes.c_int64(trg.shape[0]), _dp(src), _dp(nrm), _dp(sl),
                             _dp(dl), ctypes.c_int64(src.shape[0]), ctypes.c_double(G),
                             ctypes.c_double(nu), _dp(out))
    return out


def tri_geometry(verts, tris):
    verts = _f64(verts)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    nt = tris.shape[0]
    nrm, area, cen = np.zeros((nt, 3)), np.zeros(nt), np.zeros((nt, 3))
    _load().ko_tri_geometry(_dp(verts), tris.ctypes.data_as(_I32), ctypes.c_int64(nt), _dp(nrm),
                            _dp(area), _dp(cen))
    return nrm, area, cen


def tri_quadrature(verts, tris):
    """16 points per triangle and their weights (summing to the triangle's area)."""
    verts = _f64(verts)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    nt = tris.shape[0]
    q, w = np.zeros((16 * nt, 3)), np.zeros(16 * nt)
    _load().ko_tri_quadrature(_dp(verts), tris.ctypes.data_as(_I32), ctypes.c_int64(nt), _dp(q),
                              _dp(w))
    return q, w


def self_integrals(A, B, C, G=1.0, nu=0.3):
    """Analytic diagonal blocks at the centroid: (int U dA, PV int P dA), each 3x3."""
    A, B, C = (_f64(v).reshape(3) for v in (A, B, C))
    U, T = np.zeros(9), np.zeros(9)
    _load().ko_self_integrals(_dp(A), _dp(B), _dp(C), ctypes.c_double(G), ctypes.c_double(nu),
                              _dp(U), _dp(T))
    return U.reshape(3, 3), T.reshape(3, 3)


def bem_assemble(verts, tris, G=1.0, nu=0.3, near_levels=1):
    """Dense H = 1/2 I + P^Delta and Gm = U^Delta, (3nt) x (3nt).  near_levels > 1: the blocks
    of triangles sharing a vertex with the collocation triangle use the 4-node rule on
    4^near_levels sub-triangles (the upsampled quadrature of Sec. "Matrix-vector products")."""
    verts = _f64(verts)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    n3 = 3 * tris.shape[0]
    H, Gm = np.zeros((n3, n3)), np.zeros((n3, n3))
    _load().ko_bem_assemble_near(_dp(verts), tris.ctypes.data_as(_I32), ctypes.c_int64(tris.shape[0]),
                                 ctypes.c_double(G), ctypes.c_double(nu), ctypes.c_int(int(near_levels)), _dp(H),
                                 _dp(Gm))
    return H, Gm


def tri_block(A, B, C, x, levels=1, G=1.0, nu=0.3):
    """(int U, int T) over the triangle ABC at x by the 4-node rule on 4^levels sub-triangles."""
    A, B, C, x = (_f64(v).reshape(3) for v in (A, B, C, x))
    U, T = np.zeros(9), np.zeros(9)
    _load().ko_tri_block(_dp(A), _dp(B), _dp(C), _dp(x), ctypes.c_int(int(levels)), ctypes.c_double(G),
                         ctypes.c_double(nu), _dp(U), _dp(T))
    return U.reshape(3, 3), T.reshape(3, 3)


def bem_system(H, Gm, known_is_disp, values):
    """A x = b of Eq. num2; known_is_disp[3k+n] = 1 where u_kn is prescribed."""
    H, Gm, values = _f64(H), _f64(Gm), _f64(values).reshape(-1)
    mask = np.ascontiguousarray(known_is_disp, dtype=np.uint8).reshape(-1)
    n3 = H.shape[0]
    A, b = np.zeros((n3, n3)), np.zeros(n3)
    _load().ko_bem_system(_dp(H), _dp(Gm), ctypes.c_int64(n3), mask.ctypes.data_as(_U8),
                          _dp(values), _dp(A), _dp(b))
    return A, b


def gmres(A, b, x0=None, tol=1e-8, restart=30, maxit=1000):
    """Restarted GMRES (CGS2 Arnoldi, Givens).  Returns (x, converged, iters, relres)."""
    if restart > 255:
        raise ValueError("restart must be <= 255")
    A, b = _f64(A), _f64(b)
    x = np.zeros_like(b) if x0 is None else _f64(x0).copy()
    it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
    rc = _load().ko_gmres(_dp(A), ctypes.c_int64(b.shape[0]), _dp(b), _dp(x), ctypes.c_double(tol),
                          ctypes.c_int(restart), ctypes.c_int(maxit), ctypes.byref(it),
                          ctypes.byref(rel))
    return x, rc == 0, it.value, rel.value


def unknowns_to_fields(x, known_is_disp, values):
    """Split the Eq. num2 unknown vector back into boundary u and t, each [nt, 3]."""
    mask = np.asarray(known_is_disp, dtype=bool).reshape(-1)
    vals = np.asarray(values, dtype=np.float64).reshape(-1)
    u = np.where(mask, vals, x)
    t = np.where(mask, x, vals)
    return u.reshape(-1, 3), t.reshape(-1, 3)


def bem_interior(pts, verts, tris, u, t, G=1.0, nu=0.3, disp=True, stress=True):
    """Interior displacement [n,3] and stress [n,6] (Eq. stress_1) from the boundary solution."""
    pts, verts, u, t = _f64(pts), _f64(verts), _f64(u), _f64(t)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    n = pts.shape[0]
    dsp = np.zeros((n, 3)) if disp else None
    sig = np.zeros((n, 6)) if stress else None
    _load().ko_bem_interior(_dp(pts), ctypes.c_int64(n), _dp(verts), tris.ctypes.data_as(_I32),
                            ctypes.c_int64(tris.shape[0]), _dp(u), _dp(t), ctypes.c_double(G),
                            ctypes.c_double(nu), _dp(dsp), _dp(sig))
    return dsp, sig


def topo_derivative(sig, G=1.0, nu=0.3):
    """Eq. deriv and the energy density 1/2 sigma:eps, each [n]."""
    sig = _f64(sig).reshape(-1, 6)
    n = sig.shape[0]
    td, en = np.zeros(n), np.zeros(n)
    _load().ko_topo_derivative(_dp(sig), ctypes.c_int64(n), ctypes.c_double(G), ctypes.c_double(nu),
                               _dp(td), _dp(en))
    return td, en


def bem_solve_dense(verts, tris, known_is_disp, values, G=1.0, nu=0.3, tol=1e-8, restart=30,
                    maxit=2000):
    """Assemble, rearrange (Eq. num2) and solve with GMRES.  Returns (u, t, info)."""
    H, Gm = bem_assemble(verts, tris, G, nu)
    A, b = bem_system(H, Gm, known_is_disp, values)
    x, ok, it, rel = gmres(A, b, tol=tol, restart=restart, maxit=maxit)
    u, t = unknowns_to_fields(x, known_is_disp, values)
    return u, t, {"converged": ok, "iters": it, "relres": rel, "A": A, "b": b, "x": x}


def remove_rigid_modes(u, pts, weights=None):
    """Subtract the weighted least-squares rigid motion a + omega x p from u [n,3]."""
    u = np.asarray(u, dtype=np.float64)
    pts = np.asarray(pts, dtype=np.float64)
    w = np.ones(len(pts)) if weights is None else np.asarray(weights, dtype=np.float64)
    n = len(pts)
    M = np.zeros((3 * n, 6))
    for a in range(3):
        M[a::3, a] = 1.0
    # omega x p = [w1 p2 - w2 p1, w2 p0 - w0 p2, w0 p1 - w1 p0]
    M[0::3, 4], M[0::3, 5] = pts[:, 2], -pts[:, 1]
    M[1::3, 3], M[1::3, 5] = -pts[:, 2], pts[:, 0]
    M[2::3, 3], M[2::3, 4] = pts[:, 1], -pts[:, 0]
    sw = np.sqrt(np.repeat(w, 3))
    coef, *_ = np.linalg.lstsq(M * sw[:, None], u.reshape(-1) * sw, rcond=None)
    return (u.reshape(-1) - M @ coef).reshape(n, 3)


def periodic_U(d, G=1.0, nu=0.3, Lc=1.0, xi=0.0):
    """Periodic single-layer kernel U_per(d) of a cubic cell of side Lc (Fourier series without
    k = 0, by Ewald's split; xi <= 0 picks 4.5 / Lc) and its gradient, dU[i, j, m] = dU_ij/dd_m.
    At d = 0 (mod Lc) the regular part lim (U_per - U)."""
    d = _f64(d).reshape(3)
    U, dU = np.zeros(9), np.zeros(27)
    _load().ko_periodic_U(_dp(d), ctypes.c_double(G), ctypes.c_double(nu), ctypes.c_double(Lc),
                          ctypes.c_double(xi), _dp(U), _dp(dU))
    return U.reshape(3, 3), dU.reshape(3, 3, 3)


def periodic_disp(trg, src, nrm=None, sl=None, dl=None, G=1.0, nu=0.3, Lc=1.0, xi=0.0):
    """out[i] = sum_j U_per(x_i - y_j) sl_j + T_per(x_i - y_j, n_j) dl_j over the cubic lattice of
    side Lc (Sec. "Periodic cell of a metamaterial"); a coincident pair contributes the regular
    part of the periodic kernel."""
    trg, src, nrm, sl, dl = (_f64(a) for a in (trg, src, nrm, sl, dl))
    if dl is not None and nrm is None:
        raise ValueError("double-layer density needs normals")
    out = np.zeros((trg.shape[0], 3))
    _load().ko_periodic_disp(_dp(trg), ctypes.c_int64(trg.shape[0]), _dp(src), _dp(nrm), _dp(sl),
                             _dp(dl), ctypes.c_int64(src.shape[0]), ctypes.c_double(G),
                             ctypes.c_double(nu), ctypes.c_double(Lc), ctypes.c_double(xi), _dp(out))
    return out
