"""Multicolour hybrid Gauss-Seidel, residual, transfers, coarse solve, V-cycle.

Oracle (test infrastructure only; see the package docstring).

Paper, Sec. 4: geometric multigrid, V(3,3) cycles, a hybrid Gauss-Seidel
smoother whose lower-primitive points may be updated Jacobi-like, Gauss-Seidel
also as the coarse solver, random initial guess.  Eq. 5.1: the stencil-based
update u_I = (f_I - sum_{w != mc} s_w u_{I_w}) / s_mc.

Readings fixed here (the paper leaves them open or uses a lexicographic
order that a GPU replaces by colours):
  * one sweep = 10 steps; each step updates its node set simultaneously from
    the values at the start of the step: (1) all macro vertices; (2, 3) edge
    nodes with even / odd position p; (4-6) face nodes with (p + 2q) mod 3 =
    0, 1, 2; (7-10) cell-interior nodes with (i + 2j + 3k) mod 4 = 0..3;
    Dirichlet nodes are never updated and hold 0;
  * prolongation: a fine node that is a coarse node takes its value; every
    other fine node is the midpoint of one coarse edge and takes the mean of
    its two ends; restriction is the transpose on the unknowns; coarse
    operators are re-discretised (exact, or their own surrogate);
  * coarsest level N = 4 is solved exactly (sparse direct);
  * cycles start from u = 0 and stop at ||f - L u|| <= rtol ||f - L u0||.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import mesh as M


# ----------------------------------------------------------------------------
# Colour steps and the smoother
# ----------------------------------------------------------------------------

def colour_steps(level: M.Level):
    """The 10 node sets of one sweep (canonical indices of unknowns)."""
    N, sh = level.N, level.shell
    free = ~level.dirichlet
    steps = [np.arange(sh.nV)]
    p = np.arange(1, N)
    eidx = level.off_E + np.arange(sh.nE)[:, None] * (N - 1) + (p - 1)[None, :]
    for par in (0, 1):
        steps.append(eidx[:, p % 2 == par].ravel())
    fp = np.array([(pp, qq) for qq in range(1, N - 1) for pp in range(1, N - qq)], dtype=np.int64).reshape(-1, 2)
    nf = M.n_face_nodes(N)
    fidx = level.off_F + np.arange(sh.nF)[:, None] * nf + np.arange(nf)[None, :]
    for col in range(3):
        steps.append(fidx[:, (fp[:, 0] + 2 * fp[:, 1]) % 3 == col].ravel())
    ip = M.interior_points(N)
    nc = M.n_cell_nodes(N)
    cidx = level.off_C + np.arange(sh.nC)[:, None] * nc + np.arange(nc)[None, :]
    for col in range(4):
        steps.append(cidx[:, (ip[:, 0] + 2 * ip[:, 1] + 3 * ip[:, 2]) % 4 == col].ravel())
    return [np.sort(s[free[s]]) for s in steps]


class Operator:
    """A stencil operator on one level: the matrix over all canonical nodes,
    its diagonal and its off-diagonal part."""

    def __init__(self, level: M.Level, A: sp.csr_matrix):
        self.level = level
        self.A = A.tocsr()
        self.diag = self.A.diagonal()
        self.off = (self.A - sp.diags(self.diag)).tocsr()
        self.steps = colour_steps(level)
        self.mask = (~level.dirichlet).astype(np.float64)

    def apply(self, u):
        """y = L u on the unknowns; Dirichlet inputs read as 0, outputs are 0."""
        return self.mask * (self.A @ (self.mask * u))

    def residual(self, u, f):
        return self.mask * (f - self.A @ (self.mask * u))

    def sweep(self, u, f):
        """One multicolour hybrid Gauss-Seidel sweep (Eq. 5.1 on each step)."""
        u = self.mask * u
        for S in self.steps:
            u_new = (f[S] - self.off[S] @ u) / self.diag[S]
            u = u.copy()
            u[S] = u_new
        return u


# ----------------------------------------------------------------------------
# Transfers
# ----------------------------------------------------------------------------

def _parents(lam: np.ndarray):
    """Both coarse ends (barycentric weights on the fine lattice) of the
    coarse edge whose midpoint a fine node is; a fine node on the coarse
    lattice (all weights even) is its own parent twice."""
    odd = lam % 2 == 1
    n_odd = odd.sum(axis=1)
    d = np.zeros_like(lam)
    two = n_odd == 2
    if two.any():
        idx = np.argsort(~odd[two], axis=1, kind="stable")[:, :2]
        rows = np.flatnonzero(two)
        d[rows, idx[:, 0]] = 1
        d[rows, idx[:, 1]] = -1
    four = n_odd == 4
    if four.any():
        # (i, j, k) all odd: the coarse edge of direction (1, -1, 1), i.e. the
        # weights (lam0, lam2) move against (lam1, lam3)
        d[four] = np.array([-1, 1, -1, 1])
    return lam + d, lam - d


def prolongation(fine: M.Level, coarse: M.Level) -> sp.csr_matrix:
    """P: coarse (N/2) -> fine (N), over all canonical nodes."""
    sh, N = fine.shell, fine.N
    assert coarse.N * 2 == N
    rows, cols, vals = [], [], []

    def add(fine_idx, gids, lam, cell=None):
        a, b = _parents(lam)
        ca = M.node_index(sh, coarse.N, gids, a // 2, cell)
        cb = M.node_index(sh, coarse.N, gids, b // 2, cell)
        same = ca == cb
        rows.extend([fine_idx[same], fine_idx[~same], fine_idx[~same]])
        cols.extend([ca[same], ca[~same], cb[~same]])
        vals.extend([np.ones(same.sum()), np.full((~same).sum(), 0.5), np.full((~same).sum(), 0.5)])

    rows.append(np.arange(sh.nV))
    cols.append(np.arange(sh.nV))
    vals.append(np.ones(sh.nV))
    p = np.arange(1, N)
    for e, (a, b) in enumerate(sh.edges):
        fi = fine.off_E + e * (N - 1) + (p - 1)
        add(fi, np.tile([a, b], (N - 1, 1)), np.column_stack([N - p, p]))
    fp = np.array([(pp, qq) for qq in range(1, N - 1) for pp in range(1, N - qq)], dtype=np.int64).reshape(-1, 2)
    nf = M.n_face_nodes(N)
    if nf:
        lamf = np.column_stack([N - fp[:, 0] - fp[:, 1], fp[:, 0], fp[:, 1]])
        for f, tri in enumerate(sh.faces):
            fi = fine.off_F + f * nf + np.arange(nf)
            add(fi, np.tile(tri, (nf, 1)), lamf)
    ip = M.interior_points(N)
    nc = M.n_cell_nodes(N)
    lamc = M.cell_lambda(N, ip)
    for c in range(sh.nC):
        fi = fine.off_C + c * nc + np.arange(nc)
        add(fi, np.tile(sh.cells[c], (nc, 1)), lamc, np.full(nc, c))
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(fine.n_total, coarse.n_total))
    return P.tocsr()


class Transfer:
    def __init__(self, fine: M.Level, coarse: M.Level):
        P = prolongation(fine, coarse)
        Df = sp.diags((~fine.dirichlet).astype(np.float64))
        Dc = sp.diags((~coarse.dirichlet).astype(np.float64))
        self.P = (Df @ P @ Dc).tocsr()     # Dirichlet coarse values read as 0, fine ones written 0
        self.R = self.P.T.tocsr()

    def prolong(self, e_c):
        return self.P @ e_c

    def restrict(self, r_f):
        return self.R @ r_f


# ----------------------------------------------------------------------------
# Coarse solve and V-cycle
# ----------------------------------------------------------------------------

class CoarseSolver:
    """Exact solve on the coarsest level (the unknowns only)."""

    def __init__(self, op: Operator):
        self.op = op
        self.free = op.level.free
        self.lu = spla.splu(op.A[self.free][:, self.free].tocsc())

    def solve(self, f):
        u = np.zeros_like(f)
        u[self.free] = self.lu.solve(f[self.free])
        return u


class Hierarchy:
    """Operators on levels N = 4, 8, ..., N_fine and the transfers between
    them.  ops[0] is the coarsest (N = 4).  smooth_ops (optional, same
    levels) are the operators of the relaxation sweeps; by default the
    sweeps use ops.  Double discretisation (Sec. 4.1, "DD") relaxes with the
    surrogate and computes residuals with the exact operator: smooth_ops =
    surrogate operators, ops = exact ones."""

    def __init__(self, levels, ops, smooth_ops=None):
        self.levels = levels
        self.ops = ops
        self.smooth_ops = ops if smooth_ops is None else smooth_ops
        self.transfers = [Transfer(levels[n + 1], levels[n]) for n in range(len(levels) - 1)]
        self.coarse = CoarseSolver(ops[0])

    def vcycle(self, n, u, f, nu1=3, nu2=3):
        op, sm = self.ops[n], self.smooth_ops[n]
        if n == 0:
            return self.coarse.solve(f)
        for _ in range(nu1):
            u = sm.sweep(u, f)
        r = op.residual(u, f)
        tr = self.transfers[n - 1]
        e = self.vcycle(n - 1, np.zeros(self.levels[n - 1].n_total), tr.restrict(r), nu1, nu2)
        u = u + tr.prolong(e)
        for _ in range(nu2):
            u = sm.sweep(u, f)
        return u

    def solve_updates(self, f, u0=None, nu1=3, nu2=3, rtol=1e-8, max_cycles=50):
        """V-cycles stopped on the updates instead of the residual (the
        stopping rule Sec. 4.1 recommends for double discretisation): stop
        once ||u_k - u_{k-1}||_2 <= rtol ||u_1 - u_0||_2 (free nodes).
        Returns u and the history of relative update norms (entry 0 is 1)."""
        n = len(self.ops) - 1
        op = self.ops[n]
        u = np.zeros(self.levels[n].n_total) if u0 is None else op.mask * u0
        hist, d0 = [], None
        for _ in range(max_cycles):
            un = self.vcycle(n, u, f, nu1, nu2)
            d = np.linalg.norm((un - u)[self.levels[n].free])
            u = un
            d0 = d if d0 is None else d0
            hist.append(d / d0 if d0 > 0 else 0.0)
            if hist[-1] <= rtol:
                break
        return u, hist

    def solve(self, f, u0=None, nu1=3, nu2=3, rtol=1e-8, max_cycles=50):
        """V(nu1, nu2) cycles on the finest level; returns u and the history of
        relative residual 2-norms (entry 0 is 1)."""
        n = len(self.ops) - 1
        op = self.ops[n]
        u = np.zeros(self.levels[n].n_total) if u0 is None else op.mask * u0
        r0 = np.linalg.norm(op.residual(u, f))
        hist = [1.0]
        for _ in range(max_cycles):
            if hist[-1] <= rtol:
                break
            u = self.vcycle(n, u, f, nu1, nu2)
            hist.append(np.linalg.norm(op.residual(u, f)) / r0)
        return u, hist


def build_hierarchy(shell: M.Shell, N_fine: int, op: str = "lsqp", q: int = 2, j: int = 2,
                    mapped: bool = True):
    """Levels, operators and transfers for a shell: op = 'ifem' (exact),
    'lsqp' or 'ipoly' (surrogate of degree q on N >= 8), 'dd-lsqp' / 'dd-ipoly' (double
    discretisation: surrogate sweeps, exact residuals) or 'dd-cons' (CONS DD
    of Sec. 4.1: sweeps whose cell-interior rows are the stencils of the
    unprojected domain, exact residuals).  mapped = False builds every level
    on the unprojected domain (with 'ifem': the CONS operator)."""
    from . import fem as F
    from . import lsqp as LS
    levels, ops, sms = [], [], []
    N = 4
    while N <= N_fine:
        lv = M.make_level(shell, N, mapped=mapped)
        A = F.assemble(lv)
        S = A
        kind = op.split("-")[-1]
        if kind in ("lsqp", "ipoly") and N >= 8:
            coef = LS.fit(lv, A, q, j) if kind == "lsqp" else LS.fit_ipoly(lv, A, q=q)
            S = LS.surrogate_operator(lv, A, coef, q)
        elif kind == "cons" and N >= 8:
            lu = M.make_level(shell, N, mapped=False)
            S = LS.with_interior_stencils(lv, A, F.interior_stencils(lu, F.assemble(lu)))
        levels.append(lv)
        ops.append(Operator(lv, A if op.startswith("dd-") else S))
        sms.append(Operator(lv, S))
        N *= 2
    return Hierarchy(levels, ops, sms if op.startswith("dd-") else None)
