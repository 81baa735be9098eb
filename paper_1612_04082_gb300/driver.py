"""Topology optimisation driver (Sec. "Parallel optimization procedure").

Each iteration:
1. contours the material voxels with boundary triangles (native `voxel_surface`);
2. sets the boundary conditions;
3. solves the BVP by the FMM-accelerated BEM;
4. evaluates the topological derivative (Eq. deriv) at the centres of the material voxels;
5. removes the voxels below D_C = D_min + C (D_max - D_min) (native `voxel_threshold`);
6. post-processes the voxel array (native `voxel_clean`).

It stops when the volume ratio alpha reaches alpha_c.  The compliance Psi = 1/2 int t.u dGamma
(Eq. functional with the BEM solution) and alpha are recorded per iteration, together with the
per-element features and converged unknowns that train the learned warm start.

This module only orchestrates: every array operation of the path runs in the library (GPU
kernels for the BEM and the fields, native host code for the voxel operations).
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np

from . import (BEM_FMM, Bem, Mlp, material_K, voxel_clean, voxel_surface, voxel_threshold)

FACE_NORMALS = np.array([[-1, 0, 0], [1, 0, 0], [0, -1, 0], [0, 1, 0], [0, 0, -1], [0, 0, 1]], np.float64)


@dataclass
class Problem:
    """Voxel domain [0, nx h] x [0, ny h] x [0, nz h] with supports and loads on voxel faces."""
    nx: int
    ny: int
    nz: int
    h: float
    support: np.ndarray   # uint8 [nx, ny, nz]: voxels whose support faces are clamped (never removed)
    loaded: np.ndarray    # uint8 [nx, ny, nz]: voxels carrying the load (never removed)
    support_dir: int      # face direction (0..5) of the clamped faces
    load_dir: int         # face direction of the loaded faces
    traction: tuple = (0.0, 0.0, -1.0)
    G: float = 1.0
    nu: float = 0.3

    def frozen(self):
        return ((self.support + self.loaded) > 0).astype(np.uint8)

    def boundary_conditions(self, cell, fdir):
        """known_is_disp [nt, 3] uint8 and values [nt, 3] for the faces (cell, fdir)."""
        nt = len(cell)
        kd = np.zeros((nt, 3), np.uint8)
        vals = np.zeros((nt, 3))
        sup = (self.support.reshape(-1)[cell] > 0) & (fdir == self.support_dir)
        lod = (self.loaded.reshape(-1)[cell] > 0) & (fdir == self.load_dir)
        kd[sup] = 1
        vals[lod & ~sup] = self.traction
        return kd, vals


def cantilever(n: int, patch_half: float = 0.25) -> Problem:
    """2x1x1 box of (2n, n, n) voxels: clamped on x = 0, traction (0, 0, -1) on the x = 2 face
    within patch_half of (y, z) = (0.5, 0.5)."""
    nx, ny, nz, h = 2 * n, n, n, 1.0 / n
    sup = np.zeros((nx, ny, nz), np.uint8)
    sup[0] = 1
    lod = np.zeros_like(sup)
    c = (np.arange(n) + 0.5) * h
    sel = np.abs(c - 0.5) <= patch_half
    lod[nx - 1][np.ix_(sel, sel)] = 1
    return Problem(nx, ny, nz, h, sup, lod, 0, 1)


def bridge(n: int) -> Problem:
    """3x1x1 box of (3n, n, n) voxels: u = 0 on the bottom face z = 0 over |x - 0.15| < 0.15
    and |x - 2.85| < 0.15, traction (0, 0, -1) on the top face z = 1."""
    nx, ny, nz, h = 3 * n, n, n, 1.0 / n
    x = (np.arange(nx) + 0.5) * h
    sup = np.zeros((nx, ny, nz), np.uint8)
    sup[(np.abs(x - 0.15) < 0.15) | (np.abs(x - 2.85) < 0.15), :, 0] = 1
    lod = np.zeros_like(sup)
    lod[:, :, nz - 1] = 1
    return Problem(nx, ny, nz, h, sup, lod, 4, 5)


def triangle_geometry(V, T):
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    cr = np.cross(b - a, c - a)
    area = 0.5 * np.linalg.norm(cr, axis=1)
    return (a + b + c) / 3.0, cr / (2.0 * area[:, None]), area


@dataclass
class IterationRecord:
    """One optimisation iteration: per-element features and the converged unknowns."""
    features: np.ndarray  # [nt, 11]: centroid 3, normal 3, area 1, previous unknowns 3, local TD 1
    unknowns: np.ndarray  # [nt, 3]: converged x (u where t is prescribed, t where u is)
    face_key: np.ndarray  # [nt] int64: (cell * 6 + dir) * 4 + triangle of the face
    stats: dict = field(default_factory=dict)


def face_keys(cell, fdir):
    tri = np.arange(len(cell)) % 4  # the 4 triangles of a face are consecutive
    return (cell.astype(np.int64) * 6 + fdir.astype(np.int64)) * 4 + tri


def features_for(V, T, cell, fdir, prev: IterationRecord | None, td_prev: np.ndarray | None, prev_bem=None,
                 kd=None):
    """The 11 per-element features of the warm-start model.  The previous iterate's unknowns
    are carried over by face identity; on faces new at this iteration (exposed by removed
    voxels, so inside the previous domain) the unknown displacement is the previous
    solution's interior displacement at the centroid (by the BIE, `bem_interior`)."""
    cen, nrm, area = triangle_geometry(V, T)
    keys = face_keys(cell, fdir)
    xprev = np.zeros((len(T), 3))
    if prev is not None:
        order = np.argsort(prev.face_key)
        pos = np.searchsorted(prev.face_key[order], keys)
        pos = np.clip(pos, 0, len(order) - 1)
        hit = prev.face_key[order][pos] == keys
        xprev[hit] = prev.unknowns[order[pos[hit]]]
        new = ~hit
        if prev_bem is not None and new.any():
            pts = np.ascontiguousarray(cen[new], np.float32)
            disp = np.zeros((len(pts), 3), np.float32)
            prev_bem.interior(pts, disp=disp)
            u_new = disp.astype(np.float64)
            if kd is not None:  # components with prescribed displacement carry t, unknown here
                u_new[kd[new] > 0] = 0.0
            xprev[new] = u_new
    tdl = np.zeros(len(T)) if td_prev is None else td_prev.reshape(-1)[cell]
    return np.concatenate([cen, nrm, area[:, None], xprev, tdl[:, None]], axis=1), keys


def adaptive_td(mask, h, evaluate, C, coarse=2, band=0.01, top=0.05):
    """Two-scale sampling of the topological derivative over the material voxels (Sec.
    "Discussion and future work": a coarse grid set by the smallest feature to detect, refined
    where the threshold function differs between neighbouring cells).

    evaluate(points [m, 3] float32) -> D^T [m].  Steps:
      1. one sample per coarse cell (coarse^3 voxels): its material voxel nearest the cell's
         centre; every material voxel of the cell takes that value;
      2. threshold estimate D_C = D_min + C (D_max - D_min) from the samples;
      3. exact values at every material voxel of the cells whose threshold function (value
         below D_C + band (D_max - D_min)) differs from a face-neighbouring cell's or is set
         itself, of the cells within `top` of D_max, and of the cells on the material's
         boundary, all in one further evaluation.
    Every cell holding a voxel of the material's boundary (a face towards a void or the
    outside) is evaluated exactly as well: the shape features, and the stress concentrations
    at supports, loads and holes whose D_max sets D_C, are there.
    Returns (td [nx, ny, nz] float32, exact [nx, ny, nz] bool, evaluations)."""
    ii = np.argwhere(mask > 0)
    padded = np.pad(mask > 0, 1)
    interior = np.ones(mask.shape, bool)
    for ax in range(3):
        for step in (-1, 1):
            interior &= np.roll(padded, step, axis=ax)[1:-1, 1:-1, 1:-1]
    surface = ~interior[tuple(ii.T)]
    cells = ii // coarse
    dims = np.asarray(mask.shape) // coarse + 1
    cid = (cells[:, 0] * dims[1] + cells[:, 1]) * dims[2] + cells[:, 2]
    centre = (cells + 0.5) * coarse - 0.5
    dist = np.sum((ii - centre) ** 2, axis=1)
    order = np.lexsort((dist, cid))  # per cell, the voxel nearest its centre first
    first = order[np.r_[True, cid[order][1:] != cid[order][:-1]]]
    samples = ii[first]
    pts = np.ascontiguousarray((samples + 0.5) * h, np.float32)
    val = np.asarray(evaluate(pts), np.float32)
    ucid, inv = np.unique(cid, return_inverse=True)
    cell_val = np.zeros(len(ucid), np.float32)
    cell_val[np.searchsorted(ucid, cid[first])] = val
    dmin, dmax = float(val.min()), float(val.max())
    dc = dmin + C * (dmax - dmin)
    low = cell_val < dc + band * (dmax - dmin)
    high = cell_val >= dmax - top * (dmax - dmin)
    # threshold function differing from a face neighbour (cells looked up by id)
    cpos = np.stack(np.unravel_index(ucid, tuple(dims)), axis=1)
    refine = low | high
    surf_cells = np.unique(cid[surface])
    refine[np.searchsorted(ucid, surf_cells)] = True
    for ax in range(3):
        for step in (-1, 1):
            nb = cpos.copy()
            nb[:, ax] += step
            ok = np.all((nb >= 0) & (nb < dims), axis=1)
            nid = np.ravel_multi_index(tuple(nb[ok].T), tuple(dims))
            pos = np.searchsorted(ucid, nid)
            pos = np.clip(pos, 0, len(ucid) - 1)
            hit = ucid[pos] == nid
            idx = np.flatnonzero(ok)[hit]
            refine[idx] |= low[idx] != low[pos[hit]]
    td = np.zeros(mask.shape, np.float32)
    td[tuple(ii.T)] = cell_val[inv]
    exact = np.zeros(mask.shape, bool)
    exact[tuple(samples.T)] = True
    sel = refine[inv] & ~exact[tuple(ii.T)]
    if sel.any():
        fine = ii[sel]
        td[tuple(fine.T)] = np.asarray(evaluate(np.ascontiguousarray((fine + 0.5) * h, np.float32)), np.float32)
        exact[tuple(fine.T)] = True
    td[tuple(samples.T)] = val
    return td, exact, int(len(samples) + sel.sum())


def optimize(problem: Problem, C: float = 0.02, iters: int = 10, alpha_c: float = 0.0, p: int = 6,
             solve_kw: dict | None = None, warm_start=None, device: int = 0, verbose: bool = False,
             td_sampling: str = "full"):
    """Run the hard-kill loop.  warm_start(features [nt, 11]) -> x0 [nt, 3] or None, called
    with this iteration's features (previous unknowns carried over).  td_sampling: "full"
    (D^T at every material voxel) or "adaptive" (two-scale sampling, `adaptive_td`).  Returns
    (mask, history), history = list of IterationRecord with stats {alpha, psi, iters,
    seconds, nt, removed, td_points}."""
    kw = dict(tol=1e-6, restart=100, maxit=5000, refine=True, inner_tol=1e-3)
    if solve_kw:
        kw.update(solve_kw)
    mask = np.ones((problem.nx, problem.ny, problem.nz), np.uint8)
    n0 = mask.sum()
    frozen = problem.frozen()
    history: list[IterationRecord] = []
    td_prev = None
    prev_bem = None
    for it in range(iters):
        V, T, cell, fdir = voxel_surface(mask, problem.h)
        kd, vals = problem.boundary_conditions(cell, fdir)
        feats, keys = features_for(V, T, cell, fdir, history[-1] if history else None, td_prev, prev_bem, kd)
        if prev_bem is not None:
            prev_bem.close()
            prev_bem = None
        u, t = np.zeros((len(T), 3)), np.zeros((len(T), 3))
        b = Bem(V, T, BEM_FMM, p=p, device=device)
        b.set_material(material_K(problem.G, problem.nu), problem.G)
        b.set_bc(kd, vals)
        t0 = time.perf_counter()
        x0 = None
        if warm_start is not None:
            x0 = warm_start(feats, b) if getattr(warm_start, "uses_operator", False) else warm_start(feats)
        st = b.solve(u, t, x0=None if x0 is None else np.ascontiguousarray(x0, np.float64),
                     raise_on_fail=False, **kw)
        solve_s = time.perf_counter() - t0
        ii = np.argwhere(mask > 0)
        t1 = time.perf_counter()
        if td_sampling == "adaptive":
            def evaluate(p_):
                out = np.zeros(len(p_), np.float32)
                b.topo_derivative(p_, out)
                return out
            td_full, _, n_td = adaptive_td(mask, problem.h, evaluate, C)
            td = td_full[tuple(ii.T)]
        else:
            pts = np.ascontiguousarray((ii + 0.5) * problem.h, np.float32)
            td = np.zeros(len(pts), np.float32)
            b.topo_derivative(pts, td)
            n_td = len(pts)
        td_s = time.perf_counter() - t1
        prev_bem = b  # its solution gives the next iteration's carried-over unknowns
        x = np.where(kd > 0, t, u)
        _, _, area = triangle_geometry(V, T)
        psi = 0.5 * float(np.einsum("i,ij,ij->", area, t, u))
        alpha = float(mask.sum()) / float(n0)
        td_full = np.zeros(mask.shape, np.float32)
        td_full[tuple(ii.T)] = td
        rec = IterationRecord(feats, x, keys, {"alpha": alpha, "psi": psi, "iters": st["iters"],
                                               "outer": st["outer"], "relres": st["relres"],
                                               "converged": bool(st["converged"]), "seconds": solve_s,
                                               "x0_relres": st["x0_relres"],
                                               "nt": len(T), "warm": x0 is not None, "td_points": n_td,
                                               "td_seconds": td_s})
        history.append(rec)
        if warm_start is not None and hasattr(warm_start, "observe"):
            warm_start.observe(rec)
        if verbose:
            print(f"it {it}: nt {len(T)} alpha {alpha:.3f} psi {psi:.4e} gmres {st['iters']} "
                  f"({solve_s:.2f} s) relres {st['relres']:.1e}")
        td_prev = td_full
        if alpha <= alpha_c or it == iters - 1:
            break
        removed = voxel_threshold(mask, td_full, C, frozen)
        removed += voxel_clean(mask, problem.support, frozen)
        rec.stats["removed"] = removed
        if removed == 0:
            break
    if prev_bem is not None:
        prev_bem.close()
    return mask, history


class LearnedWarmStart:
    """Initial guesses from a network trained on the earlier iterations.

    After every iteration the (features, converged unknowns) pairs of all iterations so far
    train the network (`Mlp`, on the GPU); the next iteration's features give x0.  The
    features carry the previous iterate's unknowns over (by face identity, and on newly
    exposed faces from the previous solution's interior displacement), and the network
    predicts the change from them, trained on x - x_prev of the iterations that had a
    previous iterate.  The prediction d = net(features) is used as a search direction:
    x0 = a x_prev + g d with (a, g) minimising ||b - A x0|| for the FMM operator of the new
    problem (three operator applications).  Until it is trained it returns x_prev (nothing
    before the first iteration); a guess worse than zero is dropped by the solver.
    """

    uses_operator = True

    def __init__(self, n_hidden=256, n_layers=4, epochs=150, batch=512, lr=1e-3, seed=1612, max_rows=65536):
        self.net = Mlp(11, n_hidden, n_layers, 3, seed)
        self.kw = dict(epochs=epochs, batch=batch, lr=lr, seed=seed)
        self.max_rows = max_rows
        self.rng = np.random.default_rng(seed)
        self.X, self.Y = [], []
        self.trained = False
        self.train_stats = []

    def observe(self, rec: IterationRecord):
        if not np.any(rec.features[:, 7:10]):
            return  # first iteration: no previous iterate, nothing to learn a change from
        self.X.append(rec.features.astype(np.float32))
        self.Y.append((rec.unknowns - rec.features[:, 7:10]).astype(np.float32))
        X, Y = np.concatenate(self.X), np.concatenate(self.Y)
        if len(X) > self.max_rows:
            # the training set of one iteration is bounded: the newest iteration's rows first,
            # then a random sample of the earlier ones (the cost per iteration stays flat)
            n_new = min(len(self.X[-1]), self.max_rows)
            new = np.arange(len(X) - len(self.X[-1]), len(X))[-n_new:]
            old = self.rng.choice(len(X) - len(self.X[-1]), self.max_rows - n_new, replace=False) \
                if self.max_rows > n_new else np.zeros(0, np.int64)
            keep = np.concatenate([old, new])
            X, Y = X[keep], Y[keep]
        t0 = time.perf_counter()
        st = self.net.train(X, Y, **self.kw)
        st["seconds"] = time.perf_counter() - t0
        st["rows"] = len(X)
        self.train_stats.append(st)
        self.trained = True

    def __call__(self, feats, bem=None):
        xp = np.ascontiguousarray(feats[:, 7:10], np.float64)
        if not np.any(xp):
            return None
        if not self.trained:
            return xp.copy()
        d = np.ascontiguousarray(self.net.forward(feats.astype(np.float32)), np.float64)
        if bem is None:
            return xp + d
        rhs, ax, ad = np.zeros_like(xp), np.zeros_like(xp), np.zeros_like(xp)
        bem.rhs(rhs)
        bem.matvec(xp, ax)
        bem.matvec(d, ad)
        M = np.array([[ax.ravel() @ ax.ravel(), ax.ravel() @ ad.ravel()],
                      [ad.ravel() @ ax.ravel(), ad.ravel() @ ad.ravel()]])
        q = np.array([ax.ravel() @ rhs.ravel(), ad.ravel() @ rhs.ravel()])
        try:
            a, g = np.linalg.solve(M, q)
        except np.linalg.LinAlgError:
            a, g = 1.0, 0.0
        # keep the network's direction only when it lowers the residual by >= 10%
        r_prev = np.linalg.norm(rhs - ax)
        r_new = np.linalg.norm(rhs - a * ax - g * ad)
        if not r_new <= 0.9 * r_prev:
            a, g = 1.0, 0.0
        self.last_coef = (float(a), float(g), float(r_new / max(r_prev, 1e-300)))
        return a * xp + g * d


# --------------------------------------------------------------- periodic metamaterial cell
def periodic_cell_hole(n: int, r_c: float) -> np.ndarray:
    """Material voxels of a unit periodic cell (n^3) with a spherical hole of radius r_c at its
    centre: the initial guess of the bulk-modulus design (Sec. "Periodic cell of a
    metamaterial")."""
    c = (np.arange(n) + 0.5) / n
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    return (((X - 0.5) ** 2 + (Y - 0.5) ** 2 + (Z - 0.5) ** 2) > r_c * r_c).astype(np.uint8)


def hashin_shtrikman_bulk(phi: float, G: float = 1.0, nu: float = 0.3) -> float:
    """Upper Hashin-Shtrikman bound of the bulk modulus of a material-void composite with void
    fraction phi, over the matrix's K: 1 - phi (3K + 4G) / (4G + 3K phi)."""
    K = material_K(G, nu)
    return 1.0 - phi * (3 * K + 4 * G) / (4 * G + 3 * K * phi)


def periodic_bulk_modulus(mask: np.ndarray, G: float = 1.0, nu: float = 0.3, p: int = 6, tol: float = 1e-5,
                          device: int = 0, td: bool = False):
    """Bulk modulus of the periodic unit cell of `mask` (n^3, 1 = material) over the matrix's K.

    The unit hydrostatic macro strain eps^h = I is the homogeneous field sigma^h = 3K I plus
    the periodic fluctuation u whose tractions on the void surfaces cancel it, t = -sigma^h n
    (n out of the material): one periodic BEM solve.  The cell's mean stress is
    C : [(1 - phi) eps^h + int sym(u n) dS] (the fluctuation's face terms cancel by periodicity),
    so K_eff / K = 1 - phi + (1/3) int u . n dS, phi the void fraction.  With td, also the
    TD (Eq. deriv) of the total stress sigma^h + sigma(u) at the material voxel centres.
    Returns (K_eff / K, stats, td [n_material] or None)."""
    n = mask.shape[0]
    h = 1.0 / n
    V, T, cell, fdir = voxel_surface(mask, h, periodic=True)
    _, nrm, area = triangle_geometry(V, T)
    K = material_K(G, nu)
    vals = np.ascontiguousarray(-3.0 * K * nrm)
    t0 = time.perf_counter()
    with Bem(V, T, BEM_FMM, p=p, device=device) as b:
        b.set_material(K, G)
        b.set_periodic((0.0, 0.0, 0.0), 1.0)
        b.set_bc(np.zeros((len(T), 3), np.uint8), vals)
        u = np.zeros((len(T), 3))
        st = b.solve(u, None, tol=tol, restart=100, maxit=3000, raise_on_fail=False)
        solve_s = time.perf_counter() - t0
        out = None
        if td:
            b.set_macro_stress([3 * K, 3 * K, 3 * K, 0.0, 0.0, 0.0])
            ii = np.argwhere(mask > 0)
            out = np.zeros(len(ii), np.float32)
            b.topo_derivative(np.ascontiguousarray((ii + 0.5) * h, np.float32), out)
    phi = 1.0 - float(mask.mean())
    k = 1.0 - phi + float(np.einsum("ij,ij,i->", u, nrm, area)) / 3.0
    stats = {"phi": phi, "nt": len(T), "iters": st["iters"], "relres": st["relres"],
             "converged": bool(st["converged"]), "solve_s": solve_s, "seconds": time.perf_counter() - t0}
    return k, stats, out


def periodic_design(n: int = 64, r_c: float = 0.2, alpha_c: float = 0.7, G: float = 1.0, nu: float = 0.3,
                    p: int = 6, device: int = 0, steps: int = 1):
    """Design of a periodic cell for the largest bulk modulus (Sec. "Periodic cell of a
    metamaterial"): the cell with a spherical hole of radius r_c, the TD of the total stress
    under the hydrostatic macro strain, the material voxels of the lowest TD removed down to
    the volume fraction alpha_c: in one step (the paper's single iteration) or in `steps`
    equal steps with the TD recomputed after each; then the bulk modulus of the result against
    the Hashin-Shtrikman upper bound at that fraction."""
    mask = periodic_cell_hole(n, r_c)
    target = int(round(alpha_c * mask.size))
    first = None
    for s in range(steps):
        k, st, td = periodic_bulk_modulus(mask, G, nu, p, device=device, td=True)
        if first is None:
            first = (k, st)
        ii = np.argwhere(mask > 0)
        n_remove = (int(mask.sum()) - target) // (steps - s)
        if n_remove > 0:
            drop = ii[np.argsort(td, kind="stable")[:n_remove]]
            mask[tuple(drop.T)] = 0
    k0, s0 = first
    k1, s1, _ = periodic_bulk_modulus(mask, G, nu, p, device=device)
    return mask, {"n": n, "r_c": r_c, "alpha_c": alpha_c, "steps": steps, "alpha": float(mask.mean()),
                  "initial": {"k_over_matrix": k0, "k_over_hs": k0 / hashin_shtrikman_bulk(s0["phi"], G, nu), **s0},
                  "design": {"k_over_matrix": k1, "k_over_hs": k1 / hashin_shtrikman_bulk(s1["phi"], G, nu), **s1}}


def main(argv=None):
    """Run the loop from the command line and print one line per iteration (alpha, Psi/Psi_0,
    triangles, inner GMRES iterations, solve and D^T seconds) and a closing JSON line:

      python -m paper_1612_04082_gb300.driver --case cantilever --n 48 --iters 20 --C 0.02

    --case periodic runs the bulk-modulus design of a periodic unit cell instead (n^3 voxels,
    a spherical hole of radius --r-c, hard kill down to --alpha-c in --iters steps) and prints
    one JSON line with the initial and final bulk moduli against the Hashin-Shtrikman bound:

      python -m paper_1612_04082_gb300.driver --case periodic --n 64 --r-c 0.2 --alpha-c 0.7 --iters 1
    """
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--case", default="cantilever", choices=["cantilever", "bridge", "periodic"])
    ap.add_argument("--n", type=int, default=24, help="voxels per unit length")
    ap.add_argument("--iters", type=int, default=10)
    ap.add_argument("--C", type=float, default=0.02)
    ap.add_argument("--alpha-c", type=float, default=0.0)
    ap.add_argument("--td", default="full", choices=["full", "adaptive"])
    ap.add_argument("--warm", default="previous", choices=["none", "previous", "learned"])
    ap.add_argument("--device", type=int, default=0)
    ap.add_argument("--r-c", type=float, default=0.2, help="radius of the initial hole (periodic case)")
    a = ap.parse_args(argv)
    if a.case == "periodic":
        t0 = time.perf_counter()
        _, rec = periodic_design(n=a.n, r_c=a.r_c, alpha_c=a.alpha_c if a.alpha_c > 0 else 0.7, device=a.device,
                                 steps=max(1, a.iters))
        rec["wall_s"] = time.perf_counter() - t0
        print(json.dumps(rec))
        return
    prob = cantilever(a.n) if a.case == "cantilever" else bridge(a.n)
    warm = None
    if a.warm == "previous":
        warm = lambda f: f[:, 7:10] if np.any(f[:, 7:10]) else None  # noqa: E731
    elif a.warm == "learned":
        warm = LearnedWarmStart()
    t0 = time.perf_counter()
    mask, hist = optimize(prob, C=a.C, iters=a.iters, alpha_c=a.alpha_c, warm_start=warm, device=a.device,
                          td_sampling=a.td)
    wall = time.perf_counter() - t0
    psi0 = hist[0].stats["psi"]
    rows = []
    for k, h in enumerate(hist):
        s = h.stats
        rows.append({"it": k, "alpha": s["alpha"], "psi_ratio": s["psi"] / psi0, "nt": s["nt"], "gmres": s["iters"],
                     "outer": s["outer"], "relres": s["relres"], "solve_s": s["seconds"], "td_s": s["td_seconds"],
                     "td_points": s["td_points"], "removed": s.get("removed", 0)})
        print(f"it {k:2d}  alpha {s['alpha']:.4f}  Psi/Psi0 {s['psi'] / psi0:.4f}  nt {s['nt']:7d}  gmres {s['iters']:5d} "
              f"({s['outer']} outer, relres {s['relres']:.1e})  solve {s['seconds']:.2f} s  D^T {s['td_seconds']:.2f} s "
              f"({s['td_points']} points)", flush=True)
    print(json.dumps({"case": a.case, "voxels": [prob.nx, prob.ny, prob.nz], "h": prob.h, "C": a.C, "td": a.td,
                      "warm": a.warm, "iterations": rows, "wall_s": wall}))
    if isinstance(warm, LearnedWarmStart):
        warm.net.close()


if __name__ == "__main__":
    main()
