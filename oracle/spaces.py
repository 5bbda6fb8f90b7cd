"""Multiscale spaces V_H1 and V_H2 (Section 3).

Steps, in the paper's order:

1. Continua of each coarse block K_i (Section 3.2): the matrix K_{i,m}
   (cells where kappa equals its global minimum) and the high-conductivity
   components f_j^(i): 4-connected (edge-adjacent) components of the other
   cells of the block, ordered by their smallest cell index (row-major inside
   the block).  The NLMC auxiliary functions are their indicators, eqs.
   (3.4)-(3.5).
2. CEM enrichment (Section 3.1): the auxiliary eigenproblem eq. (3.1),
   int_{K_i} kappa grad psi . grad v = lambda s_i(psi, v),
   s_i(u, v) = int_{K_i} kappa_tilde u v, kappa_tilde = kappa H^-2, with Q1
   on all nodes of the closed block (pure Neumann).  The J+1 smallest
   eigenpairs are kept; when the next eigenvalue ties the last kept one
   (gap <= 1e-8 |lambda| + 1e-12 lambda_max) the whole cluster is kept.
   Their span is projected s-orthogonally off the indicator span; directions
   whose projected s-norm^2 is below 1e-8 (the constant) are dropped.  The
   remaining J_i enrichment functions are made canonical: s-orthonormal,
   rotated to the eigenvectors of the nodal weight
   w(x,y) = x + 0.6180339887 y + 0.3 x^2 - 0.2 y^3 + 0.1 x y applied to their
   nodal part (x, y block-local in [0,1]), ascending, each signed so that
   sum_nodes exp(x + 1.7 y) e(x,y) > 0 over its nodal part.
   V_aux^(i) = span{indicators} + span{enrichment}.
3. Constraint energy minimising bases on K_i^+ (eq. (3.2)):
   a(phi, v) + s(mu, v) = 0 for all v in V_0(K_i^+),
   s(phi, nu) = s(psi, nu) for all nu in V_aux(K_i^+).
   K_i^+ is K_i enlarged by ell coarse layers, clipped at the domain; phi
   vanishes on its boundary; mu ranges over V_aux(K_i^+) (the printed
   "mu in V(K_i^+)" is read as a typo).  With psi an indicator this is the
   NLMC problem eq. (3.6), its integral constraints rescaled to
   kappa_tilde-weighted averages so that each basis takes the value ~1 on
   its own continuum (then the sum of all NLMC bases is a partition of unity
   and psi_bar of eq. (3.7) is the smooth "constant basis" Section 3.2
   describes).  Solved here as one sparse KKT system per window.
4. eq. (3.7): psi_bar = (1/L) sum of the fracture bases, L = sum_i m_i the
   number of fracture bases (the printed inner sum from m = 0 would also
   add the matrix bases; with them the first L-1 psi_tilde sum to a vector
   lying almost in V_H2 and gamma -> 1, while with the fracture bases alone
   the L psi_tilde sum to exactly zero, the linear dependency that dropping
   the last basis removes); psi_tilde = psi - s(psi, psi_bar) /
   s(psi_bar, psi_bar) psi_bar for the fracture and enrichment bases;
   V_H1 = their span without the last fracture basis; V_H2 =
   span{psi_bar, psi_0^(i)}.  With no fracture at all (L = 0) there is no
   psi_bar: V_H1 is the enrichment and V_H2 = span{psi_0^(i)}.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import K_REF, M_REF, FineProblem

CLUSTER_REL = 1e-8
CLUSTER_ABS = 1e-12
ENRICH_DROP = 1e-8


def ritz_weight(xl, yl):
    return xl + 0.6180339887 * yl + 0.3 * xl * xl - 0.2 * yl ** 3 + 0.1 * xl * yl


def sign_weight(xl, yl):
    return np.exp(xl + 1.7 * yl)


def components(mask: np.ndarray):
    """4-connected components of True cells; each a sorted list of flat cell
    indices, components ordered by their smallest index."""
    ny, nx = mask.shape
    label = -np.ones(mask.shape, dtype=np.int64)
    comps = []
    for start in range(nx * ny):
        sy, sx = divmod(start, nx)
        if not mask[sy, sx] or label[sy, sx] >= 0:
            continue
        cid = len(comps)
        stack = [(sy, sx)]
        label[sy, sx] = cid
        cells = []
        while stack:
            y, x = stack.pop()
            cells.append(y * nx + x)
            for yy, xx in ((y - 1, x), (y + 1, x), (y, x - 1), (y, x + 1)):
                if 0 <= yy < ny and 0 <= xx < nx and mask[yy, xx] and label[yy, xx] < 0:
                    label[yy, xx] = cid
                    stack.append((yy, xx))
        comps.append(sorted(cells))
    return comps


class Block:
    """Closed coarse block (bx, by): bs x bs cells, (bs+1)^2 local nodes
    (local node (a, b) has id b*(bs+1) + a)."""

    def __init__(self, fp: FineProblem, bx: int, by: int, J: int):
        n_f, nc = fp.n_f, fp.nc
        bs = n_f // nc
        self.bx, self.by, self.bs = bx, by, bs
        h = 1.0 / n_f
        self.h = h
        a, b = np.meshgrid(np.arange(bs + 1), np.arange(bs + 1))
        a = a.ravel()
        b = b.ravel()
        self.gid = (by * bs + b) * (n_f + 1) + (bx * bs + a)
        self.xl = a / bs
        self.yl = b / bs
        nb = (bs + 1) ** 2
        self.nb = nb
        kap = fp.kappa[by * bs:(by + 1) * bs, bx * bs:(bx + 1) * bs]
        kt = fp.kappa_tilde[by * bs:(by + 1) * bs, bx * bs:(bx + 1) * bs]
        A = np.zeros((nb, nb))
        S = np.zeros((nb, nb))
        corners = []
        for cj in range(bs):
            for ci in range(bs):
                cor = [cj * (bs + 1) + ci, cj * (bs + 1) + ci + 1,
                       (cj + 1) * (bs + 1) + ci + 1, (cj + 1) * (bs + 1) + ci]
                corners.append(cor)
                A[np.ix_(cor, cor)] += kap[cj, ci] * K_REF
                S[np.ix_(cor, cor)] += kt[cj, ci] * h * h * M_REF
        self.A, self.S = A, S
        self.corners = np.array(corners)
        ktf = kt.ravel()
        # -- step 1: continua and their indicator functionals ----------------
        matrix = (kap == fp.kappa.min())
        conts = []
        if matrix.any():
            conts.append(np.nonzero(matrix.ravel())[0])
        self.has_matrix = bool(matrix.any())
        fr = components(~matrix)
        conts.extend(np.array(c) for c in fr)
        self.n_frac = len(fr)
        R = np.zeros((len(conts), nb))       # r_C . phi = s(phi, chi_C)
        G = np.zeros(len(conts))             # s(chi_C, chi_C)
        for q, cells in enumerate(conts):
            for c in cells:
                R[q, self.corners[c]] += ktf[c] * h * h / 4.0
                G[q] += ktf[c] * h * h
        self.R, self.G = R, G
        # -- step 2: CEM eigen-enrichment ------------------------------------
        lam, vec = sla.eigh(A, S)
        self.lam = lam
        n_sel = min(J + 1, nb) if J > 0 else 0
        lmax = abs(lam[-1])
        while 0 < n_sel < nb and (lam[n_sel] - lam[n_sel - 1]
                                  <= CLUSTER_REL * abs(lam[n_sel]) + CLUSTER_ABS * lmax):
            n_sel += 1
        V = vec[:, :n_sel]
        self.V = V
        if n_sel > 0:
            RV = R @ V
            Gp = np.eye(n_sel) - RV.T @ (RV / G[:, None])
            sig, U = np.linalg.eigh(0.5 * (Gp + Gp.T))
            keep = sig > ENRICH_DROP
            C0 = U[:, keep] / np.sqrt(sig[keep])[None, :]
            if C0.shape[1] > 0:
                Vn = V @ C0
                Rw = Vn.T @ (ritz_weight(self.xl, self.yl)[:, None] * Vn)
                _, E = np.linalg.eigh(0.5 * (Rw + Rw.T))
                Cc = C0 @ E
                sg = np.sign(sign_weight(self.xl, self.yl) @ (V @ Cc))
                sg[sg == 0] = 1.0
                Cc = Cc * sg[None, :]
            else:
                Cc = C0
        else:
            Cc = np.zeros((0, 0))
        self.Cc = Cc                          # enrichment coefficients in V
        self.n_enr = Cc.shape[1]
        # constraint rows of the block's aux basis: [indicators..., enrichment...]
        rows = [R[q] for q in range(R.shape[0])]
        gdiag = list(G)
        for k in range(self.n_enr):
            nod = V @ Cc[:, k]
            a_c = (R @ nod) / G
            rows.append(S @ nod - a_c @ R)
            gdiag.append(1.0)
        self.con_rows = np.array(rows).reshape(len(rows), nb)
        self.con_gram = np.array(gdiag)       # s(nu_k, nu_k), the basis is s-orthogonal
        # kinds of this block's bases: 0 matrix, 1 fracture, 2 enrichment
        self.kinds = ([0] if self.has_matrix else []) + [1] * self.n_frac + [2] * self.n_enr


class Window:
    """Oversampled region K_i^+ of block (bx, by): ell coarse layers, clipped;
    unknowns are the nodes strictly inside the window rectangle."""

    def __init__(self, fp: FineProblem, bx: int, by: int, ell: int):
        nc, n_f = fp.nc, fp.n_f
        bs = n_f // nc
        self.bx0, self.bx1 = max(0, bx - ell), min(nc - 1, bx + ell)
        self.by0, self.by1 = max(0, by - ell), min(nc - 1, by + ell)
        X0, X1 = self.bx0 * bs, (self.bx1 + 1) * bs
        Y0, Y1 = self.by0 * bs, (self.by1 + 1) * bs
        i, j = np.meshgrid(np.arange(X0 + 1, X1), np.arange(Y0 + 1, Y1))
        self.gid = (j * (n_f + 1) + i).ravel()
        self.blocks = [(x, y) for y in range(self.by0, self.by1 + 1)
                       for x in range(self.bx0, self.bx1 + 1)]


def cem_window(fp: FineProblem, blocks: dict, win: Window, target):
    """eq. (3.2) on one window for every auxiliary function of the target
    block (sparse KKT system, direct solve).  Returns [n_window, n_target]."""
    gid = win.gid
    loc = -np.ones((fp.n_f + 1) ** 2, dtype=np.int64)
    loc[gid] = np.arange(gid.size)
    Aw = fp.A_full[gid][:, gid]
    rr, cc, vv = [], [], []
    r = 0
    t0 = None
    for key in win.blocks:
        blk = blocks[key]
        li = loc[blk.gid]
        keep = np.nonzero(li >= 0)[0]
        for q in range(blk.con_rows.shape[0]):
            rr.extend([r] * keep.size)
            cc.extend(li[keep].tolist())
            vv.extend(blk.con_rows[q, keep].tolist())
            if key == target and q == 0:
                t0 = r
            r += 1
    m = r
    C = sp.csr_matrix((vv, (rr, cc)), shape=(m, gid.size))
    K = sp.bmat([[Aw, C.T], [C, None]], format="csc")
    tb = blocks[target]
    nt = tb.con_rows.shape[0]
    rhs = np.zeros((gid.size + m, nt))
    for q in range(nt):
        rhs[gid.size + t0 + q, q] = tb.con_gram[q]
    # Sparse LU of the indefinite KKT matrix, then two steps of iterative
    # refinement with the same factors: at contrast 1e6 the plain solve leaves
    # forward errors up to ~1e-9 of the basis values (residuals ~1e-14), which
    # refinement removes, so the bases meet the FP64 accuracy eq. (3.2) asks of
    # the reduced model.
    lu = spla.splu(K)
    sol = lu.solve(rhs)
    for _ in range(2):
        sol += lu.solve(rhs - K @ sol)
    return sol[:gid.size, :]


def default_workers() -> int:
    """Host threads for the independent per-block and per-window problems."""
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:
        return max(1, os.cpu_count() or 1)


def _map(fn, items, workers):
    """[fn(x) for x in items], in order; the blocks and windows are
    independent problems, so they may run on several threads (SciPy's sparse
    LU and LAPACK release the GIL).  The result does not depend on workers."""
    if workers <= 1 or len(items) <= 1:
        return [fn(x) for x in items]
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, items))


class Spaces:
    """All bases and the V_H1 / V_H2 split for one FineProblem."""

    def __init__(self, fp: FineProblem, J: int, ell: int, workers: int | None = None):
        self.fp = fp
        nc = fp.nc
        self.J, self.ell = J, ell
        workers = default_workers() if workers is None else workers
        keys = [(bx, by) for by in range(nc) for bx in range(nc)]
        self.blocks = dict(zip(keys, _map(lambda k: Block(fp, k[0], k[1], J), keys, workers)))
        gpos = -np.ones((fp.n_f + 1) ** 2, dtype=np.int64)
        gpos[fp.interior] = np.arange(fp.D)
        wins = {k: Window(fp, k[0], k[1], ell) for k in keys}
        phis = _map(lambda k: cem_window(fp, self.blocks, wins[k], k), keys, workers)
        cols, kind, owner = [], [], []
        for (bx, by), phi in zip(keys, phis):
            full = np.zeros((fp.D, phi.shape[1]))
            full[gpos[wins[(bx, by)].gid], :] = phi
            cols.extend(full[:, c] for c in range(phi.shape[1]))
            kind.extend(self.blocks[(bx, by)].kinds)
            owner.extend([by * nc + bx] * phi.shape[1])
        self.Psi_all = np.column_stack(cols)
        self.kind = np.array(kind)
        self.owner = np.array(owner)
        self._split()

    def _split(self):
        fp = self.fp
        P = self.Psi_all
        mt = np.nonzero(self.kind == 0)[0]
        fr = np.nonzero(self.kind == 1)[0]
        h1 = np.nonzero(self.kind >= 1)[0]          # fracture + enrichment, in order
        L = fr.size
        self.L = L
        if L > 0:
            psi_bar = P[:, fr].sum(axis=1) / L
            Sb = fp.S @ psi_bar
            coef = (Sb @ P[:, h1]) / (psi_bar @ Sb)
            tilde = P[:, h1] - np.outer(psi_bar, coef)
            drop = np.nonzero(h1 == fr[-1])[0][0]
            keep = np.ones(h1.size, dtype=bool)
            keep[drop] = False
            self.Psi1 = tilde[:, keep]
            self.Psi2 = np.column_stack([psi_bar, P[:, mt]])
            self.psi_bar = psi_bar
        else:
            self.Psi1 = P[:, h1]
            self.Psi2 = P[:, mt]
            self.psi_bar = None
        self.d1 = self.Psi1.shape[1]
        self.d2 = self.Psi2.shape[1]
