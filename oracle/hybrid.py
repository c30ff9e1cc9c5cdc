"""Plain FP64 CPU oracle of the hybrid FEM/FDM scheme (arXiv 1509.01399).

TEST INFRASTRUCTURE ONLY.  This package exists to check the CUDA path; only
``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs
of ``bench.py`` may import it.  It shares no code with the CUDA library and
never calls it.

What it computes, in the paper's order and notation (numpy / scipy.sparse,
float64 throughout):

* Mesh (Sec. 7.1, Sec. 3): a structured lattice of nodes
  x = origin + (dx_1 i, dx_2 j, dx_3 k) (one spacing h on every axis, or the
  steps dx_1, dx_2, dx_3 of the 7-point Laplacian of Sec. 7.3); a
  finite-element block of nodes lo..hi whose voxels (bricks) are each cut into
  the six Kuhn tetrahedra along the voxel diagonal; the node classes of Algorithm 1:
  omega_o (the block's boundary shell, owned by the FDM), omega_diamond (the
  next shell inward, owned by the FEM), omega_* (the FEM interior) and
  omega_+ (every other lattice node, FDM).
* FEM operators (Sec. 7.1-7.2): element mass and stiffness of P1 functions,
  M^K_ij = (phi_i, phi_j)_K and K^K_ij = (a_h grad phi_i, grad phi_j)_K, with
  the mass matrix lumped by rows and the coefficient a_h piecewise constant
  (Eq. (p0)), one value per voxel.  The explicit scheme is Eq. (fem):
  u^{k+1} = (2 - tau^2 (M^L)^{-1} K) u^k - u^{k-1} (the G term only acts on
  rows of nodes on the FEM block boundary, which Algorithm 1 overwrites from
  the FDM, so it never reaches an owned row).
* FDM (Sec. 7.3): the leapfrog Eq. (fdmschemeforward) with the 7-point
  Laplacian (a second difference over dx_d^2 per axis d); Neumann faces by a
  mirror ghost; the plane-wave source d_n u = p(t) of Model Problem 2
  (Eq. (model2), Eq. (f)) by the ghost u_g = u_in + 2 h p (h the spacing
  normal to the face).
* Absorbing faces (Sec. 7.4): Eq. (eq:abs2),
  u_b^{k+1} = u_{b1}^k + r u_b^k - r u_{b1}^{k+1},  r = (h - tau) / (h + tau)
  with h the spacing normal to the face, applied after the interior rows of
  the same time level; a node on several absorbing faces takes the mean of
  its per-face formulas, faces before edges before corners.
* Algorithm 2 (Sec. 7.5): per time step, update the FDM-owned rows, update
  the FEM-owned rows, copy omega_diamond from FEM to FDM and omega_o from FDM
  to FEM, swap levels.
* Adjoint and gradient (Sec. 6, Eq. (lagrangian1) - Eq. (grad1new),
  Eq. (gradient1)): the exact discrete adjoint of the time stepping, obtained
  by writing each step as E_k u^{k+1} = B_k u^k - C_k u^{k-1} + s_k and
  transposing those matrices literally; the conductivity gradient is
  dJ/da_c = -tau^2 sum_k (lambda^{k+1})^T (M^L)^{-1} K_c u^k, the discrete
  form of int_0^T grad u . grad lambda dt.
* Tikhonov functional (Eq. (functional)) and one conjugate-gradient update of
  Algorithm 3 (Sec. 8) with a quadratic-fit step length.
* The telegraph reading u_tt + sigma u_t - div grad u = 0 (a = 1, sigma on the
  unknown voxels): the damping lumped like the mass and central in time, its
  exact discrete adjoint and the gradient with respect to sigma.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

BC_NEUMANN0 = 0
BC_ABC = 1


def p1_element(X: np.ndarray):
    """Volumes and barycentric gradients of P1 tetrahedra.

    X: (T, 4, 3) vertex coordinates.  Returns vol (T,) and grads (T, 4, 3)
    where grads[t, i] = grad phi_i on tetrahedron t (Sec. 7.2: the P1 basis
    functions of the reference element mapped by F_K)."""
    T = X.shape[0]
    A = np.concatenate([np.ones((T, 4, 1)), X], axis=2)  # rows: (1, x_v)
    Ainv = np.linalg.inv(A)  # column i holds the coefficients of phi_i
    grads = np.transpose(Ainv[:, 1:, :], (0, 2, 1))
    e = X[:, 1:, :] - X[:, :1, :]
    vol = np.abs(np.linalg.det(e)) / 6.0
    return vol, grads


def element_stiffness(vol, grads, a_tet):
    """K^K_ij = a_K |K| grad phi_i . grad phi_j (Sec. 7.2)."""
    return (a_tet * vol)[:, None, None] * np.einsum("tid,tjd->tij", grads, grads)


def kuhn_tets(origin_nodes: np.ndarray):
    """The six Kuhn tetrahedra of a unit voxel with corner `origin_nodes`
    (V, 3) lattice coordinates: each is the path 0 -> e_p -> e_p + e_q -> (1,1,1)
    for a permutation (p, q, s) of the axes.  Returns (V, 6, 4, 3)."""
    V = origin_nodes.shape[0]
    out = np.zeros((V, 6, 4, 3), dtype=np.int64)
    for t, perm in enumerate(itertools.permutations(range(3))):
        v = np.zeros(3, dtype=np.int64)
        out[:, t, 0] = origin_nodes
        for s in range(3):
            v[perm[s]] = 1
            out[:, t, s + 1] = origin_nodes + v
    return out


def refine_voxels(tet_nodes, tet_unknown, refine, n_lattice):
    """Refine the marked voxels once by bisection.  The refinement edge of a
    Kuhn tetrahedron v0 v1 v2 v3 (v0, v3 the voxel's diagonal corners) is the
    diagonal v0 v3, shared by the six tetrahedra of the voxel and by no other
    voxel; bisecting it at the voxel centre c replaces each tetrahedron by
    (v0, v1, v2, c) and (c, v1, v2, v3).  The mesh stays conforming.  Centre
    nodes get the ids n_lattice, n_lattice + 1, ... in unknown-voxel order."""
    cid = np.full(refine.size, -1, dtype=np.int64)
    cid[refine] = n_lattice + np.arange(int(refine.sum()))
    keep = (tet_unknown < 0) | ~refine[np.maximum(tet_unknown, 0)]
    par = ~keep
    pn = tet_nodes[par]
    pu = tet_unknown[par]
    c = cid[pu]
    ch1 = np.stack([pn[:, 0], pn[:, 1], pn[:, 2], c], axis=1)
    ch2 = np.stack([c, pn[:, 1], pn[:, 2], pn[:, 3]], axis=1)
    nodes = np.concatenate([tet_nodes[keep], ch1, ch2], axis=0)
    unk = np.concatenate([tet_unknown[keep], pu, pu])
    return nodes, unk, cid


@dataclass
class Phase:
    """Boundary state of the step leaving t_k: the absorbing faces in force and
    the faces that carry the plane-wave flux (Neumann faces with d_n u = g)."""

    abc_faces: tuple
    src_faces: tuple
    t: float


def pulse(omega: float, s):
    """p(s) = sin(omega s) on [0, t1], t1 = 2 pi / omega, and 0 elsewhere
    (Eq. (f)); s may be an array."""
    s = np.asarray(s, dtype=np.float64)
    t1 = 2.0 * math.pi / omega
    return np.where((s >= 0.0) & (s <= t1), np.sin(omega * s), 0.0)


class Problem:
    """Lattice, FEM block, node classes and assembled operators."""

    def __init__(self, n, h, fem_lo=None, fem_hi=None, bc=(BC_ABC,) * 6, origin=(0.0, 0.0, 0.0), refine=None):
        """h: one spacing for every axis, or the three steps (dx_1, dx_2, dx_3)
        of Sec. 7.3 (then `h` is None and `hv` holds them).  refine: optional
        boolean per unknown voxel (x fastest); each marked voxel is refined
        once by bisection (see `refine_voxels`)."""
        self.n = tuple(int(v) for v in n)
        if min(self.n) < 3:
            raise ValueError("every axis needs at least 3 nodes")
        hv = np.asarray(h, dtype=np.float64)
        self.hv = np.full(3, float(hv)) if hv.ndim == 0 else np.array(hv, dtype=np.float64).reshape(3)
        if not (self.hv > 0).all():
            raise ValueError("spacings must be > 0")
        self.iso = bool(self.hv[0] == self.hv[1] == self.hv[2])
        self.h = float(self.hv[0]) if self.iso else None
        self.bc = tuple(int(b) for b in bc)
        self.origin = tuple(float(o) for o in origin)
        nx, ny, nz = self.n
        self.N = nx * ny * nz
        kk, jj, ii = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        self.I = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
        self.on_face = []
        for f in range(6):
            ax, side = divmod(f, 2)
            self.on_face.append(self.I[:, ax] == (0 if side == 0 else self.n[ax] - 1))
        self.stride = (1, nx, nx * ny)

        self.has_fem = fem_lo is not None
        if self.has_fem:
            lo = np.array(fem_lo, dtype=np.int64)
            hi = np.array(fem_hi, dtype=np.int64)
            if (lo < 0).any() or (hi > np.array(self.n) - 1).any() or (hi - lo < 2).any():
                raise ValueError("bad FEM block")
            self.lo, self.hi = lo, hi
            in_box = np.all((self.I >= lo) & (self.I <= hi), axis=1)
            self.owned = np.all((self.I >= lo + 1) & (self.I <= hi - 1), axis=1)
            inner = np.all((self.I >= lo + 2) & (self.I <= hi - 2), axis=1)
            self.omega_o = in_box & ~self.owned
            self.omega_diamond = self.owned & ~inner
            # voxels of the FEM block and their Kuhn tetrahedra
            cz, cy, cx = np.meshgrid(*[np.arange(lo[d], hi[d]) for d in (2, 1, 0)], indexing="ij")
            vox = np.stack([cx.ravel(), cy.ravel(), cz.ravel()], axis=1)
            unk = np.all((vox >= lo + 1) & (vox <= hi - 2), axis=1)
            ud = np.maximum(hi - lo - 2, 0)
            self.unknown_dims = tuple(int(v) for v in ud)
            self.n_unknown = int(np.prod(ud))
            uid = np.full(vox.shape[0], -1, dtype=np.int64)
            rel = vox[unk] - (lo + 1)
            uid[unk] = rel[:, 0] + ud[0] * (rel[:, 1] + ud[1] * rel[:, 2])
            tets = kuhn_tets(vox)  # (V, 6, 4, 3)
            tet_nodes = self.node_id(tets.reshape(-1, 3)).reshape(-1, 4)
            tet_unknown = np.repeat(uid, 6)
            X_all = self.I.astype(np.float64) * self.hv
            self.NC = 0
            self.center_of_unknown = np.full(self.n_unknown, -1, dtype=np.int64)
            if refine is not None and self.n_unknown:
                refine = np.asarray(refine, dtype=bool).ravel()
                if refine.size != self.n_unknown:
                    raise ValueError("refine mask must have one entry per unknown voxel")
                tet_nodes, tet_unknown, centres = refine_voxels(tet_nodes, tet_unknown, refine, self.N)
                self.NC = int(refine.sum())
                self.center_of_unknown[np.flatnonzero(refine)] = self.N + np.arange(self.NC)
                rel_ids = np.flatnonzero(refine)
                cvox = np.stack([rel_ids % ud[0], (rel_ids // ud[0]) % ud[1], rel_ids // (ud[0] * ud[1])], axis=1)
                X_all = np.concatenate([X_all, (cvox + lo + 1 + 0.5) * self.hv], axis=0)
            self.tet_nodes = tet_nodes
            self.tet_unknown = tet_unknown
            self.tet_vol, self.tet_grads = p1_element(X_all[tet_nodes])
            self.voxel_volume = self.cell_volume()
        else:
            self.owned = np.zeros(self.N, dtype=bool)
            self.omega_o = np.zeros(self.N, dtype=bool)
            self.omega_diamond = np.zeros(self.N, dtype=bool)
            self.unknown_dims = (0, 0, 0)
            self.n_unknown = 0
            self.voxel_volume = self.cell_volume()
            self.NC = 0
        # state vectors hold the lattice nodes, then the refinement centres
        self.NT = self.N + self.NC
        pad = np.zeros(self.NC, dtype=bool)
        self.owned = np.concatenate([self.owned, np.ones(self.NC, dtype=bool)])
        self.omega_o = np.concatenate([self.omega_o, pad])
        self.omega_diamond = np.concatenate([self.omega_diamond, pad])
        self.on_face = [np.concatenate([f, pad]) for f in self.on_face]
        self.fdm_owned = ~self.owned
        self.owned_nodes = np.flatnonzero(self.owned)
        self.owned_pos = np.full(self.NT, -1, dtype=np.int64)
        self.owned_pos[self.owned_nodes] = np.arange(self.owned_nodes.size)
        self.D = self._fdm_laplacian()
        self._phase_cache = {}

    # ------------------------------------------------------------------ mesh
    def cell_volume(self):
        """Volume of one lattice cell: h^3, or dx_1 dx_2 dx_3."""
        return self.h ** 3 if self.iso else float(self.hv[0] * self.hv[1] * self.hv[2])

    def r_abc(self, dt):
        """r = (h - tau) / (h + tau) of Eq. (eq:abs2) per axis, h the spacing
        normal to the face."""
        return (self.hv - dt) / (self.hv + dt)

    def node_id(self, ijk):
        ijk = np.asarray(ijk, dtype=np.int64)
        return ijk[..., 0] + self.n[0] * (ijk[..., 1] + self.n[1] * ijk[..., 2])

    def face_nodes(self, f):
        """Nodes of face f in trace order: the two in-face axes p < q, index
        = c_p + n_p * c_q."""
        ax = f // 2
        p, q = [d for d in range(3) if d != ax]
        nodes = np.flatnonzero(self.on_face[f])
        key = self.I[nodes, p] + self.n[p] * self.I[nodes, q]
        return nodes[np.argsort(key, kind="stable")]

    def face_weights(self, f):
        """Lumped surface quadrature weight of each face node: the in-face cell
        area (h^2, or dx_p dx_q for the face's axes p, q) halved for every
        in-face coordinate that sits on the face's own border."""
        nodes = self.face_nodes(f)
        ax = f // 2
        p, q = [d for d in range(3) if d != ax]
        w = np.full(nodes.size, self.h ** 2 if self.iso else float(self.hv[p] * self.hv[q]))
        for d in range(3):
            if d == ax:
                continue
            edge = (self.I[nodes, d] == 0) | (self.I[nodes, d] == self.n[d] - 1)
            w[edge] *= 0.5
        return w

    # ------------------------------------------------------------- operators
    def _fdm_laplacian(self):
        """7-point Delta_h of Sec. 7.3 on every lattice node (the second
        difference along axis d over dx_d^2), Neumann mirror ghost
        u_{-1} = u_{1} on the outer faces (the ghost values of source faces add
        a constant, handled in the source term)."""
        rows, cols, vals = [], [], []
        ids = np.arange(self.N)
        for d in range(3):
            inv_h2 = 1.0 / self.hv[d] ** 2
            c = self.I[:, d]
            st = self.stride[d]
            lowb = c == 0
            highb = c == self.n[d] - 1
            mid = ~lowb & ~highb
            rows += [ids[mid], ids[mid], ids[lowb], ids[highb]]
            cols += [ids[mid] - st, ids[mid] + st, ids[lowb] + st, ids[highb] - st]
            vals += [np.full(mid.sum(), inv_h2), np.full(mid.sum(), inv_h2),
                     np.full(lowb.sum(), 2 * inv_h2), np.full(highb.sum(), 2 * inv_h2)]
            rows.append(ids)
            cols.append(ids)
            vals.append(np.full(self.N, -2 * inv_h2))
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.NT, self.NT))

    def tet_coefficient(self, a_unknown):
        """a_K per tetrahedron: the voxel's value on unknown voxels, 1 on the
        other voxels of the FEM block (a = 1 near Omega_FDM, Eq. (2.3))."""
        a_unknown = np.asarray(a_unknown, dtype=np.float64)
        a_tet = np.ones(self.tet_nodes.shape[0])
        m = self.tet_unknown >= 0
        a_tet[m] = a_unknown[self.tet_unknown[m]]
        return a_tet

    def assemble(self, a_unknown):
        """Global stiffness K(a) and lumped mass M^L over the FEM block."""
        if not self.has_fem:
            return sp.csr_matrix((self.NT, self.NT)), np.zeros(self.NT)
        Kloc = element_stiffness(self.tet_vol, self.tet_grads, self.tet_coefficient(a_unknown))
        r = np.repeat(self.tet_nodes, 4, axis=1).ravel()
        c = np.tile(self.tet_nodes, (1, 4)).ravel()
        K = sp.csr_matrix((Kloc.ravel(), (r, c)), shape=(self.NT, self.NT))
        ML = np.bincount(self.tet_nodes.ravel(), weights=np.repeat(self.tet_vol / 4.0, 4),
                         minlength=self.NT)
        return K, ML

    def space_operator(self, a_unknown):
        """L such that a non-absorbing row reads u^{k+1} = 2u^k - u^{k-1} - tau^2 (L u^k)_i:
        -Delta_h on FDM-owned rows, (M^L)^{-1} K on FEM-owned rows."""
        K, ML = self.assemble(a_unknown)
        inv_ml = np.zeros(self.NT)
        inv_ml[self.owned] = 1.0 / ML[self.owned]
        Lfe = sp.diags(inv_ml) @ K
        Lfd = -self.D
        return (sp.diags(self.fdm_owned.astype(float)) @ Lfd + sp.diags(self.owned.astype(float)) @ Lfe).tocsr()

    # ----------------------------------------------------------------- phase
    def plane_wave(self, src):
        """Geometry of the plane wave u = F(t - d.(x - x0)) that the source
        launches: unit direction d (for a face source, d = -n of its face, the
        wave of Model Problem 2), entry corner x0 (lattice index: the corner
        where d.x is smallest) and the faces it enters through, each with the
        factor -(d . n_f) > 0 of its Neumann flux
        d_n u = -(d . n_f) p(t - d.(x - x0)) (Eq. (f) written for an oblique
        incidence; for d = -n it is d_n u = p(t) of Eq. (model2))."""
        d = getattr(src, "direction", None)
        if d is None:
            ax, side = divmod(src.face, 2)
            d = np.zeros(3)
            d[ax] = 1.0 if side == 0 else -1.0
        d = np.asarray(d, dtype=np.float64)
        d = d / math.sqrt(float(np.dot(d, d)))
        i0 = [0 if d[ax] >= 0.0 else self.n[ax] - 1 for ax in range(3)]
        entry = {}
        for f in range(6):
            ax, side = divmod(f, 2)
            dn = d[ax] * (-1.0 if side == 0 else 1.0)
            if dn < 0.0:
                entry[f] = -dn
        return d, i0, entry

    def switch_time(self, src, f):
        """Last instant at which entry face f carries the flux: t1 plus the
        largest delay d.(x - x0) over the face (t1 for a face source)."""
        d, i0, _ = self.plane_wave(src)
        ax = f // 2
        p, q = [b for b in range(3) if b != ax]
        if self.iso:
            return 2.0 * math.pi / src.omega + self.h * (abs(d[p]) * (self.n[p] - 1) + abs(d[q]) * (self.n[q] - 1))
        return 2.0 * math.pi / src.omega + (abs(d[p]) * (self.n[p] - 1) * self.hv[p] +
                                            abs(d[q]) * (self.n[q] - 1) * self.hv[q])

    def phase(self, src, k, dt):
        """Boundary state for the step from t_k = k dt: an entry face of the
        source acts as a Neumann face with the plane-wave flux while
        t_k <= its switch time, and takes the mesh's own condition afterwards
        (Model Problem 2: S_{1,1} then S_{1,2})."""
        abc = [f for f in range(6) if self.bc[f] == BC_ABC]
        t = k * dt
        srcf = []
        if src is not None:
            _, _, entry = self.plane_wave(src)
            srcf = [f for f in sorted(entry) if t <= self.switch_time(src, f)]
            abc = [f for f in abc if f not in srcf]
        return Phase(tuple(abc), tuple(srcf), t)

    def source_term(self, src, ph: Phase, dt):
        """s with s_i = tau^2 (2 / h) g_i on the non-absorbing nodes of the
        flux faces (h the spacing normal to the face): the mirror ghost
        u_g = u_in + 2 h g of d_n u = g, summed over the flux faces a node lies
        on; g = amp (-(d . n_f)) p(t_k - d.(x_i - x0))."""
        s = np.zeros(self.NT)
        if not ph.src_faces:
            return s
        d, i0, entry = self.plane_wave(src)
        level, _ = self.abc_structure(ph.abc_faces)
        if self.iso:
            delay = self.h * (d[0] * (self.I[:, 0] - i0[0]) + d[1] * (self.I[:, 1] - i0[1]) +
                              d[2] * (self.I[:, 2] - i0[2]))
        else:
            delay = (d[0] * self.hv[0] * (self.I[:, 0] - i0[0]) + d[1] * self.hv[1] * (self.I[:, 1] - i0[1]) +
                     d[2] * self.hv[2] * (self.I[:, 2] - i0[2]))
        p = pulse(src.omega, ph.t - delay)
        for f in ph.src_faces:
            m = self.on_face[f][: self.N] & (level[: self.N] == 0)
            s[: self.N][m] += dt * dt * 2.0 / self.hv[f // 2] * src.amp * entry[f] * p[m]
        return s

    def abc_structure(self, abc_faces):
        """Level (number of absorbing faces a node lies on) and, per absorbing
        face, its nodes b with the inward neighbours b1 and the face's axis."""
        key = tuple(abc_faces)
        if key in self._phase_cache:
            return self._phase_cache[key]
        level = np.zeros(self.NT, dtype=np.int64)
        for f in abc_faces:
            level += self.on_face[f]
        pairs = []
        for f in abc_faces:
            ax, side = divmod(f, 2)
            b = np.flatnonzero(self.on_face[f])
            b1 = b + (self.stride[ax] if side == 0 else -self.stride[ax])
            pairs.append((b, b1, ax))
        self._phase_cache[key] = (level, pairs)
        return level, pairs

    def abc_self(self, level, pairs, r):
        """Coefficient of u_b^k in the absorbing row of node b: r, or on
        anisotropic lattices the mean of the r of the node's absorbing faces."""
        if self.iso:
            return np.full(self.NT, r[0])
        acc = np.zeros(self.NT)
        for b, _, ax in pairs:
            acc[b] += r[ax]
        return acc / np.maximum(level, 1)

    def step_matrices(self, Lop, phase: Phase, dt):
        """E, B, C of one step written as E u^{k+1} = B u^k - C u^{k-1} + s
        (the source vector s is `source_term`)."""
        level, pairs = self.abc_structure(phase.abc_faces)
        r = self.r_abc(dt)
        rself = self.abc_self(level, pairs, r)
        nonabc = (level == 0).astype(float)
        I = sp.identity(self.NT, format="csr")
        Dn = sp.diags(nonabc)
        B = Dn @ (2.0 * I - dt * dt * Lop)
        E = Dn @ I
        C = Dn @ I
        rb, cb, vb, ve = [], [], [], []
        abcn = np.flatnonzero(level > 0)
        rb.append(abcn)
        cb.append(abcn)
        vb.append(rself[abcn])
        ve.append(np.ones(abcn.size))
        for b, b1, ax in pairs:
            Lb = level[b].astype(float)
            rb.append(b)
            cb.append(b1)
            vb.append(1.0 / Lb)
            ve.append(r[ax] / Lb)
        rr, cc = np.concatenate(rb), np.concatenate(cb)
        B = (B + sp.csr_matrix((np.concatenate(vb), (rr, cc)), shape=B.shape)).tocsr()
        E = (E + sp.csr_matrix((np.concatenate(ve), (rr, cc)), shape=E.shape)).tocsr()
        return E, B, C.tocsr()

    # --------------------------------------------------------------- forward
    def forward(self, a_unknown, src, nsteps, dt, init=None, keep_hist=False, keep_fields=False, damp=None):
        """Algorithm 2, forward in time, with separate FDM and FEM arrays and
        the two copies of Algorithm 1 per step.  damp: the telegraph reading's
        s_i = tau D_i / (2 M^L_i) per node (see `damping_ratio`), which turns
        the FEM rows into (1 + s) u^{k+1} = 2 u^k - (1 - s) u^{k-1} - tau^2 (M^L)^{-1} K u^k.

        Returns a dict with the trace on the source face (rows t_0 .. t_N),
        the final level u^N (and u^{N-1}), optionally u^k on the FEM-owned
        nodes for k = 0 .. N-1 (for the gradient) and every full level."""
        tau2 = dt * dt
        r = self.r_abc(dt)
        K, ML = self.assemble(a_unknown)
        own = self.owned
        obs = self.face_nodes(src.face) if src is not None else np.zeros(0, dtype=np.int64)
        if init is None:
            u_fd = np.zeros(self.NT)
            u_fd_prev = np.zeros(self.NT)
        else:
            u_fd = np.array(init[0], dtype=np.float64)
            u_fd_prev = np.array(init[1], dtype=np.float64)
        u_fe, u_fe_prev = u_fd.copy(), u_fd_prev.copy()
        trace = np.zeros((nsteps + 1, obs.size))
        trace[0] = u_fd[obs]
        hist = np.zeros((nsteps, self.owned_nodes.size)) if keep_hist else None
        fields = [self._combine(u_fd, u_fe)] if keep_fields else None
        for k in range(nsteps):
            if keep_hist:
                hist[k] = u_fe[self.owned_nodes]
            ph = self.phase(src, k, dt)
            level, pairs = self.abc_structure(ph.abc_faces)
            # 1. FDM rows at omega_+ and omega_o (non-absorbing rows)
            rows = self.fdm_owned & (level == 0)
            lap = self.D @ u_fd
            new_fd = np.zeros(self.NT)
            new_fd[rows] = 2.0 * u_fd[rows] - u_fd_prev[rows] + tau2 * lap[rows]
            if ph.src_faces:
                new_fd[rows] += self.source_term(src, ph, dt)[rows]
            # 2. FEM rows at omega_* and omega_diamond, Eq. (fem)
            new_fe = np.zeros(self.NT)
            if self.has_fem:
                Ku = K @ u_fe
                if damp is None:
                    new_fe[own] = 2.0 * u_fe[own] - u_fe_prev[own] - tau2 * Ku[own] / ML[own]
                else:
                    so = damp[own]
                    new_fe[own] = (2.0 * u_fe[own] - (1.0 - so) * u_fe_prev[own] - tau2 * Ku[own] / ML[own]) / (1.0 + so)
                # 3. FEM values at omega_diamond become FDM boundary values
                new_fd[self.omega_diamond] = new_fe[self.omega_diamond]
            # absorbing rows, Eq. (eq:abs2), faces before edges before corners
            rself = self.abc_self(level, pairs, r)
            for L in (1, 2, 3):
                acc = None
                for b, b1, ax in pairs:
                    sel = level[b] == L
                    if not sel.any():
                        continue
                    bb, bb1 = b[sel], b1[sel]
                    if acc is None:
                        acc = np.zeros(self.NT)
                    acc[bb] += u_fd[bb1] - r[ax] * new_fd[bb1]
                if acc is not None:
                    m = level == L
                    new_fd[m] = rself[m] * u_fd[m] + acc[m] / L
            if self.has_fem:
                # 4. FDM values at omega_o become FEM boundary values
                new_fe[self.omega_o] = new_fd[self.omega_o]
            # 5. swap
            u_fd_prev, u_fd = u_fd, new_fd
            u_fe_prev, u_fe = u_fe, new_fe
            trace[k + 1] = u_fd[obs]
            if keep_fields:
                fields.append(self._combine(u_fd, u_fe))
        return dict(trace=trace, u=self._combine(u_fd, u_fe), u_prev=self._combine(u_fd_prev, u_fe_prev),
                    hist=hist, fields=fields)

    def _combine(self, u_fd, u_fe):
        u = u_fd.copy()
        u[self.owned] = u_fe[self.owned]
        return u

    # ------------------------------------------------- matrix form and adjoint
    def operators(self, a_unknown, src, nsteps, dt):
        """Step matrices for every distinct boundary phase of the run."""
        Lop = self.space_operator(a_unknown)
        cache = {}
        seq = []
        for k in range(nsteps + 2):
            ph = self.phase(src, k, dt)
            key = (ph.abc_faces, ph.src_faces)
            if key not in cache:
                cache[key] = self.step_matrices(Lop, ph, dt)
            seq.append((key, ph))
        return cache, seq

    @staticmethod
    def _strict_part(E, transpose=False):
        Nm = (E - sp.identity(E.shape[0], format="csr")).tocsr()
        Nm.eliminate_zeros()
        return Nm.T.tocsr() if transpose else Nm

    @staticmethod
    def _solve_unit(Nm, y):
        """Solve (I + N) x = y, where N only couples a node on l absorbing
        faces to nodes on l - 1 of them (or the transpose of that): N is
        nilpotent with N^4 = 0, so the fixed point x = y - N x is exact after
        4 sweeps."""
        x = y.copy()
        for _ in range(4):
            x = y - Nm @ x
        return x

    def forward_matrix(self, a_unknown, src, nsteps, dt, forcing=None, init=None):
        """The same time stepping as `forward`, written as
        E_k u^{k+1} = B_k u^k - C_k u^{k-1} + s_k (+ f_k); returns the trace."""
        cache, seq = self.operators(a_unknown, src, nsteps, dt)
        obs = self.face_nodes(src.face)
        u = np.zeros(self.NT) if init is None else np.array(init[0], dtype=np.float64)
        up = np.zeros(self.NT) if init is None else np.array(init[1], dtype=np.float64)
        trace = np.zeros((nsteps + 1, obs.size))
        trace[0] = u[obs]
        strict = {key: self._strict_part(E) for key, (E, _, _) in cache.items()}
        for k in range(nsteps):
            key, ph = seq[k]
            E, B, C = cache[key]
            y = B @ u - C @ up + self.source_term(src, ph, dt)
            if forcing is not None:
                y = y + forcing[k]
            un = self._solve_unit(strict[key], y)
            up, u = u, un
            trace[k + 1] = u[obs]
        return trace, u

    def adjoint(self, a_unknown, src, nsteps, dt, cot, hist, return_lambda=False, keep_lambdas=False):
        """Exact discrete adjoint, backward in time:
        E_{j-1}^T lambda^j = B_j^T lambda^{j+1} - C_{j+1}^T lambda^{j+2} + c^j,
        j = N .. 1, lambda^{N+1} = lambda^{N+2} = 0, where c^j is dJ/du^j
        (non-zero on the observation face only).  Returns dJ/da per unknown
        voxel: -tau^2 sum_k (lambda^{k+1})^T (M^L)^{-1} K_c u^k."""
        cache, seq = self.operators(a_unknown, src, nsteps, dt)
        K, ML = self.assemble(a_unknown)
        obs = self.face_nodes(src.face)
        lam1 = np.zeros(self.NT)
        lam2 = np.zeros(self.NT)
        Gacc = np.zeros(self.n_unknown)
        lams = [None] * (nsteps + 2) if keep_lambdas else None
        tr = {key: (self._strict_part(E, transpose=True), B.T.tocsr(), C.T.tocsr())
              for key, (E, B, C) in cache.items()}
        for j in range(nsteps, 0, -1):
            _, BT, _ = tr[seq[j][0]]
            _, _, CT = tr[seq[j + 1][0]]
            NT, _, _ = tr[seq[j - 1][0]]
            rhs = BT @ lam1 - CT @ lam2
            rhs[obs] += cot[j]
            lam = self._solve_unit(NT, rhs)
            if j <= nsteps - 1 and self.n_unknown:
                Gacc += self.pair(hist[j], lam1, ML)
            lam2, lam1 = lam1, lam
            if keep_lambdas:
                lams[j] = lam
        if self.n_unknown:
            Gacc += self.pair(hist[0], lam1, ML)
        out = -dt * dt * Gacc
        if keep_lambdas:
            return out, lams
        if return_lambda:
            return out, lam1
        return out

    def lumped_mass(self, a_unknown):
        """Diagonal mass M in which the hybrid operator is symmetric: on
        FDM-owned rows the lumped lattice mass (the cell volume), halved for
        every axis on which the node lies on the outer boundary; on FEM-owned
        rows the lumped finite-element mass M^L (Sec. 7.2)."""
        M = np.full(self.NT, self.cell_volume())
        for d in range(3):
            b = np.concatenate([(self.I[:, d] == 0) | (self.I[:, d] == self.n[d] - 1), np.zeros(self.NC, dtype=bool)])
            M[b] *= 0.5
        if self.has_fem:
            _, ML = self.assemble(a_unknown)
            M[self.owned] = ML[self.owned]
        return M

    def adjoint_paper(self, a_unknown, src, nsteps, dt, cot, hist, return_lambda=False):
        """The paper's adjoint, solved backward in time by Algorithm 2 with
        separate FDM and FEM arrays: Eq. (fdmschemeadjoint) on the FDM-owned
        rows and the second line of Eq. (fem) on the FEM-owned rows,
        lambda^{k-1} = 2 lambda^k - lambda^{k+1} + tau^2 Delta_h lambda^k + s^k,
        from lambda^N = lambda^{N+1} = 0 (Eq. (adjoint1): lambda(T) =
        lambda_t(T) = 0), with d_n lambda = 0 (mirror ghost) on every face.
        The data residual enters on S_T as the mirror ghost of the flux
        d_n lambda = -(u - u~) z_delta that Eq. (control1) puts there: with the
        cotangent c^k = dJ/d(trace row k) = w_k m_j (u - u~), s^k_j = -tau c^k_j / M_j.
        Returns g_c = tau sum_k int_c grad u^k . grad lambda^k (Eq. (gradient1),
        same time index), the paper's approximation of dJ/da_c."""
        tau2 = dt * dt
        K, ML = self.assemble(a_unknown)
        M = self.lumped_mass(a_unknown)
        own = self.owned
        obs = self.face_nodes(src.face)
        ones = np.ones(self.NT)
        lam_fd, lam_fd_next = np.zeros(self.NT), np.zeros(self.NT)   # lambda^k, lambda^{k+1}
        lam_fe, lam_fe_next = np.zeros(self.NT), np.zeros(self.NT)
        G = np.zeros(self.n_unknown)
        for k in range(nsteps, 0, -1):
            if k <= nsteps - 1 and self.n_unknown:
                G += self.pair(hist[k], self._combine(lam_fd, lam_fe), ones)
            # 1. FDM rows, Eq. (fdmschemeadjoint), Neumann ghosts on every face
            rows = self.fdm_owned
            new_fd = np.zeros(self.NT)
            new_fd[rows] = 2.0 * lam_fd[rows] - lam_fd_next[rows] + tau2 * (self.D @ lam_fd)[rows]
            new_fd[obs] += -dt * cot[k] / M[obs]
            # 2. FEM rows, Eq. (fem) second line (the G term never reaches an owned row)
            new_fe = np.zeros(self.NT)
            if self.has_fem:
                new_fe[own] = 2.0 * lam_fe[own] - lam_fe_next[own] - tau2 * (K @ lam_fe)[own] / ML[own]
                # 3.-4. exchange of Algorithm 1 / Algorithm 2
                new_fd[self.omega_diamond] = new_fe[self.omega_diamond]
                new_fe[self.omega_o] = new_fd[self.omega_o]
            # 5. swap
            lam_fd_next, lam_fd = lam_fd, new_fd
            lam_fe_next, lam_fe = lam_fe, new_fe
        lam0 = self._combine(lam_fd, lam_fe)
        if self.n_unknown:
            G += self.pair(hist[0], lam0, ones)
        out = dt * G
        return (out, lam0) if return_lambda else out

    def pair(self, u_owned, lam, ML):
        """Per unknown voxel c: (lambda / M^L)^T K_c u = sum over the voxel's
        tetrahedra of |K| grad u . grad (lambda / M^L), with K_c the a = 1
        stiffness of the voxel."""
        m = self.tet_unknown >= 0
        tn = self.tet_nodes[m]
        uK = u_owned[self.owned_pos[tn]]
        lhat = lam / np.where(ML > 0, ML, 1.0)
        lK = lhat[tn]
        gu = np.einsum("ti,tid->td", uK, self.tet_grads[m])
        gl = np.einsum("ti,tid->td", lK, self.tet_grads[m])
        val = self.tet_vol[m] * np.sum(gu * gl, axis=1)
        return np.bincount(self.tet_unknown[m], weights=val, minlength=self.n_unknown)


# ------------------------------------------------------------ functional, CG
def data_weights(prob: Problem, face: int, nsteps: int, dt: float, mode: str = "plain"):
    """Weights of the misfit 1/2 int_{S_T} (u - u~)^2 z_delta (Eq. (functional)).

    'plain': 1/2 sum_{k>=1} sum_j (u - u~)^2 (the plain least-squares loss);
    'quadrature': time weight tau for k >= 1 and the lumped face weight of
    each node."""
    wk = np.ones(nsteps + 1)
    wk[0] = 0.0
    if mode == "plain":
        return wk, np.ones(prob.face_nodes(face).size)
    if mode == "quadrature":
        return wk * dt, prob.face_weights(face)
    raise ValueError(mode)


def misfit(trace, obs, wk, mj):
    d = trace - obs
    return 0.5 * float(np.sum(wk[:, None] * mj[None, :] * d * d)), wk[:, None] * mj[None, :] * d


def value_and_grad(prob: Problem, a, sources, nsteps, dt, obs_traces, gamma=0.0, a0=1.0,
                   mode="plain", need_grad=True, adjoint="exact", init=None):
    """F(a) = sum over sources of the data misfit + gamma/2 sum_c |c| (a_c - a0)^2
    and its Euclidean gradient dF/da_c (Eq. (functional), Eq. (grad1new)):
    adjoint='exact' by the discrete adjoint, 'paper' by the paper's adjoint
    scheme (`Problem.adjoint_paper`).  init: (u^0, u^{-1}) of Model Problem 1
    (Eq. (model1)), the same for every source; None: Model Problem 2."""
    J = 0.5 * gamma * prob.voxel_volume * float(np.sum((a - a0) ** 2))
    g = gamma * prob.voxel_volume * (a - a0)
    traces = []
    for s, src in enumerate(sources):
        res = prob.forward(a, src, nsteps, dt, keep_hist=need_grad, init=init)
        wk, mj = data_weights(prob, src.face, nsteps, dt, mode)
        Jd, cot = misfit(res["trace"], obs_traces[s], wk, mj)
        J += Jd
        traces.append(res["trace"])
        if need_grad:
            adj = prob.adjoint if adjoint == "exact" else prob.adjoint_paper
            g = g + adj(a, src, nsteps, dt, cot, res["hist"])
    return J, (g if need_grad else None), traces


def quadratic_step(J0, dJ0, alpha_t, Jt):
    """Step length from the parabola through J(0), J'(0) and J(alpha_t),
    clamped to [0, 4 alpha_t]; alpha_t itself when the parabola has no
    minimum.  (Algorithm 3 leaves the step-size rule open.)"""
    curv = Jt - J0 - dJ0 * alpha_t
    if curv <= 0.0:
        alpha = alpha_t
    else:
        alpha = -dJ0 * alpha_t * alpha_t / (2.0 * curv)
    return min(max(alpha, 0.0), 4.0 * alpha_t)


def projected_gradient(a, g, a_min, a_max):
    """g with the components zeroed on voxels that sit at a bound of the
    admissible set [a_min, a_max] (Eq. (admpar)) and whose gradient points out
    of it (a = a_min with g > 0, a = a_max with g < 0): the projection clips
    those components, so they can neither move nor lower F."""
    blocked = ((a <= a_min) & (g > 0.0)) | ((a >= a_max) & (g < 0.0))
    return np.where(blocked, 0.0, g)


def drop_blocked(a, d, a_min, a_max):
    """d with the components zeroed that would leave [a_min, a_max] at once
    (a = a_min with d < 0, a = a_max with d > 0)."""
    blocked = ((a <= a_min) & (d < 0.0)) | ((a >= a_max) & (d > 0.0))
    return np.where(blocked, 0.0, d)


def cg_direction(g, d_prev, gn2_prev, vol):
    """Fletcher-Reeves direction of Algorithm 3, Step 2: d^m = -g^m + beta^m d^{m-1},
    beta^m = ||g^m||^2 / ||g^{m-1}||^2 (L2 norms over the unknown voxels),
    d^0 = -g^0."""
    gn2 = vol * float(np.sum(g * g))
    if d_prev is None or gn2_prev is None or gn2_prev <= 0.0:
        return -g, 0.0, gn2
    beta = gn2 / gn2_prev
    return -g + beta * d_prev, beta, gn2


def cg_step(prob: Problem, a, sources, nsteps, dt, obs_traces, state: dict, gamma=0.01, a0=1.0,
            a_min=1.0, a_max=5.0, mode="quadrature"):
    """One iteration of Algorithm 3 on the admissible set [a_min, a_max]
    (Eq. (admpar)): state and adjoint at a^m (Step 1); the gradient
    g^m = int grad u . grad lambda dt + gamma (a^m - a0) as an L2 function on
    the voxels; the Fletcher-Reeves update (Step 2) of the projected gradient
    (`projected_gradient`), with the components of d^m that the projection
    would clip at once dropped and a restart d^m = -g^m when d^m is not a
    descent direction; the step length from the parabola through F(0), F'(0)
    and F at a trial step; projection a^{m+1} = clip(a^m + alpha d^m).

    The trial step is 0.5 / max|d^m| at the first iteration and whenever the
    previous step failed to lower F (or was 0), else the previous step
    length.  state: d, gn2 (||projected g^{m-1}||^2), alpha, J (F(a^{m-1})),
    iter.  Returns (a^{m+1}, state, report); report['gnorm'] is ||g^m||_L2,
    the stopping measure of Step 3."""
    vol = prob.voxel_volume
    J0, ge, _ = value_and_grad(prob, a, sources, nsteps, dt, obs_traces, gamma, a0, mode)
    g = ge / vol
    gp = projected_gradient(a, g, a_min, a_max)
    d, beta, gn2 = cg_direction(gp, state.get("d"), state.get("gn2"), vol)
    d = drop_blocked(a, d, a_min, a_max)
    dJ0 = float(np.sum(ge * d))
    if dJ0 >= 0.0:
        d, beta = -gp, 0.0
        dJ0 = float(np.sum(ge * d))
    alpha_prev, J_prev = state.get("alpha"), state.get("J")
    if alpha_prev is None or alpha_prev <= 0.0 or (J_prev is not None and J0 >= J_prev):
        alpha_t = 0.5 / max(float(np.max(np.abs(d))), 1e-300)
    else:
        alpha_t = alpha_prev
    a_t = np.clip(a + alpha_t * d, a_min, a_max)
    Jt, _, _ = value_and_grad(prob, a_t, sources, nsteps, dt, obs_traces, gamma, a0, mode, need_grad=False)
    alpha = quadratic_step(J0, dJ0, alpha_t, Jt)
    a_new = np.clip(a + alpha * d, a_min, a_max)
    new_state = dict(d=d, gn2=gn2, alpha=alpha, J=J0, iter=state.get("iter", 0) + 1)
    report = dict(J=J0, gnorm=math.sqrt(vol * float(np.sum(g * g))), gpnorm=math.sqrt(gn2), alpha=alpha,
                  beta=beta, dJ0=dJ0, J_trial=Jt, alpha_trial=alpha_t)
    return a_new, new_state, report


# ------------------------------------------------------ telegraph reading
# u_tt + sigma u_t - div grad u = 0 (the damped reading of the model, with
# a = 1 and the unknown sigma >= 0 on the unknown voxels, 0 elsewhere).  The
# damping term is discretised like the mass: central in time,
# D (u^{k+1} - u^{k-1}) / (2 tau) with D lumped by rows over the Kuhn
# tetrahedra of the voxels carrying sigma.
def damping_weights(prob: Problem):
    """W (unknown voxels x nodes): W[v, i] = the lumped mass voxel v gives
    node i, |K| / 4 summed over v's tetrahedra with i as a vertex, so that
    the lumped damping is D = W^T sigma."""
    m = prob.tet_unknown >= 0
    rows = np.repeat(prob.tet_unknown[m], 4)
    cols = prob.tet_nodes[m].ravel()
    vals = np.repeat(prob.tet_vol[m] / 4.0, 4)
    return sp.csr_matrix((vals, (rows, cols)), shape=(prob.n_unknown, prob.NT))


def damping_ratio(prob: Problem, sigma, dt):
    """s_i = tau D_i / (2 M^L_i) on the FEM-owned rows (0 elsewhere)."""
    _, ML = prob.assemble(np.ones(prob.n_unknown))
    D = damping_weights(prob).T @ np.asarray(sigma, dtype=np.float64)
    s = np.zeros(prob.NT)
    own = prob.owned
    s[own] = 0.5 * dt * D[own] / ML[own]
    return s


def telegraph_forward(prob: Problem, sigma, src, nsteps, dt, init=None, keep_levels=False):
    """The forward of the telegraph reading (Algorithm 2 with the damped FEM
    rows).  keep_levels: also the FEM-owned values of u^{-1} .. u^N (rows
    0 .. N + 1), which the sigma-gradient pairs."""
    s = damping_ratio(prob, sigma, dt)
    res = prob.forward(np.ones(prob.n_unknown), src, nsteps, dt, init=init, keep_hist=keep_levels, damp=s)
    if keep_levels:
        own = prob.owned_nodes
        first = np.zeros(own.size) if init is None else np.asarray(init[1], dtype=np.float64)[own]
        res["levels"] = np.vstack([first[None, :], res["hist"], res["u"][own][None, :]])
    return res


def telegraph_adjoint(prob: Problem, sigma, src, nsteps, dt, cot, levels):
    """Exact discrete adjoint of the damped recursion, written per step as
    E_k u^{k+1} = B_k u^k - C_k u^{k-1} + s_k with E_k = E_k^0 + S and
    C_k = C_k^0 - S (S = diag(s), the undamped matrices of `step_matrices`):
    E_{j-1}^T lambda^j = B_j^T lambda^{j+1} - C_{j+1}^T lambda^{j+2} + c^j.
    Returns dJ/dsigma_v = -sum_k (lambda^{k+1})^T (dS/dsigma_v) (u^{k+1} - u^{k-1})
    with dS_ii/dsigma_v = tau W[v, i] / (2 M^L_i)."""
    s = damping_ratio(prob, sigma, dt)
    S = sp.diags(s)
    Lop = prob.space_operator(np.ones(prob.n_unknown))
    _, ML = prob.assemble(np.ones(prob.n_unknown))
    cache, seq = {}, []
    for k in range(nsteps + 2):
        ph = prob.phase(src, k, dt)
        key = (ph.abc_faces, ph.src_faces)
        if key not in cache:
            E, B, C = prob.step_matrices(Lop, ph, dt)
            Et = (E + S).T.tocsr()
            dg = Et.diagonal()
            Nt = (Et - sp.diags(dg)).tocsr()
            Nt.eliminate_zeros()
            cache[key] = (Nt, dg, B.T.tocsr(), (C - S).T.tocsr())
        seq.append(key)
    obs = prob.face_nodes(src.face)
    Wd = damping_weights(prob)
    scale = np.zeros(prob.NT)
    scale[prob.owned] = 0.5 * dt / ML[prob.owned]
    own = prob.owned_nodes
    lam1 = np.zeros(prob.NT)
    lam2 = np.zeros(prob.NT)
    G = np.zeros(prob.n_unknown)

    def pair(k, lam):  # (lambda^{k+1})^T (dS/dsigma) (u^{k+1} - u^{k-1}), all voxels
        v = np.zeros(prob.NT)
        v[own] = levels[k + 2] - levels[k]
        return Wd @ (scale * lam * v)

    for j in range(nsteps, 0, -1):
        _, _, BT, _ = cache[seq[j]]
        _, _, _, CT = cache[seq[j + 1]]
        Nt, dg, _, _ = cache[seq[j - 1]]
        rhs = BT @ lam1 - CT @ lam2
        rhs[obs] += cot[j]
        lam = rhs / dg  # (D + N)^T x = y by the fixed point x = (y - N^T x) / D: N couples
        for _ in range(4):  # absorbing rows only (where D = 1) and is nilpotent
            lam = (rhs - Nt @ lam) / dg
        if j <= nsteps - 1 and prob.n_unknown:
            G -= pair(j, lam1)
        lam2, lam1 = lam1, lam
    if prob.n_unknown:
        G -= pair(0, lam1)
    return G


def telegraph_value_and_grad(prob: Problem, sigma, sources, nsteps, dt, obs_traces, mode="plain", init=None):
    """Data misfit of the telegraph reading summed over sources, and its
    gradient with respect to sigma on the unknown voxels."""
    J = 0.0
    g = np.zeros(prob.n_unknown)
    traces = []
    for s_, src in enumerate(sources):
        res = telegraph_forward(prob, sigma, src, nsteps, dt, init=init, keep_levels=True)
        wk, mj = data_weights(prob, src.face, nsteps, dt, mode)
        Jd, cot = misfit(res["trace"], obs_traces[s_], wk, mj)
        J += Jd
        traces.append(res["trace"])
        g = g + telegraph_adjoint(prob, sigma, src, nsteps, dt, cot, res["levels"])
    return J, g, traces


def problem_from_workload(w) -> Problem:
    refine = getattr(w, "refine", None)
    spacing = getattr(w, "spacing", None)
    return Problem(w.n, w.h if spacing is None else spacing, w.fem_lo, w.fem_hi, w.bc, w.origin, refine=refine)
