"""Helpers of the sampled parity tests (no tests here).

* `lower_sample`: a few hundred vertex / edge / face nodes on the boundaries
  of a few seeded macro cells, so that the oracle's single-cell row assembly
  (oracle.local.node_rows) touches a bounded number of cells even on the
  3840-cell shells.
* `step_of`: the smoother step (0..9) of canonical nodes (the 10-step sweep:
  vertices; edge nodes by parity of their position p; face nodes by
  (p + 2q) mod 3; cell interiors by (i + 2j + 3k) mod 4).
* Per-node FP32 error bounds.  With eps = 2^-23 and the FP64 oracle's
  result x on the same FP32-rounded inputs:
    apply     |y_I - x_I| <= C eps sum_w |s_w u_w|
    residual  |r_I - x_I| <= C eps (sum_w |s_w u_w| + |f_I|)
    smoother  |u_I - x_I| <= C eps (sum_{w != mc} |s_w x_w| + |f_I|) / |s_mc|
  Each FP32 update is a sum of 15 products whose weights come from a short
  FP32 polynomial evaluation (a few roundings each, no cancellation to speak
  of: the weights vary by a few per cent over a cell), so one update carries
  about 20 eps of the sum of absolute terms; within a sweep an update also
  inherits its neighbours' errors weighted by |s_w| / |s_mc| (sum about 1),
  so errors add over the colour steps.  C = 64 covers one sweep's 10 steps
  and C = 128 two sweeps.
"""
from __future__ import annotations

import numpy as np

from oracle import local as LO
from oracle import mesh as M

EPS32 = 2.0 ** -23


def lower_sample(sh, N, cells, per_cell, seed, vertices=True):
    """Non-Dirichlet vertex, edge and face nodes on the boundaries of `cells`:
    up to `per_cell` of each cell's boundary edge/face nodes (seeded), and,
    with `vertices`, the cell's first vertex."""
    off_E = M.offsets(sh, N)[0]
    off_C = M.offsets(sh, N)[2]
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for c in cells:
        cm = LO.cell_map(sh, N, int(c))
        bnd = np.unique(cm[(cm < off_C) & (cm >= off_E)])
        bnd = bnd[~M.dirichlet_of(sh, N, bnd)]
        out.append(rng.choice(bnd, size=min(per_cell, len(bnd)), replace=False))
        if vertices:
            v = np.array([int(sh.cells[int(c)][0])])
            out.append(v[~M.dirichlet_of(sh, N, v)])
    return np.unique(np.concatenate(out))


def step_of(sh, N, idx):
    """Smoother step (0..9) of canonical nodes idx (array)."""
    off_E, off_F, off_C, _ = M.offsets(sh, N)
    idx = np.asarray(idx, dtype=np.int64)
    out = np.empty(len(idx), dtype=np.int64)
    v = idx < off_E
    out[v] = 0
    e = (idx >= off_E) & (idx < off_F)
    p = (idx[e] - off_E) % (N - 1) + 1
    out[e] = 1 + (p % 2)
    f = (idx >= off_F) & (idx < off_C)
    fp = np.array([(pp, qq) for qq in range(1, N - 1) for pp in range(1, N - qq)], dtype=np.int64).reshape(-1, 2)
    loc = (idx[f] - off_F) % M.n_face_nodes(N)
    out[f] = 3 + (fp[loc, 0] + 2 * fp[loc, 1]) % 3
    c = idx >= off_C
    ip = M.interior_points(N)[(idx[c] - off_C) % M.n_cell_nodes(N)]
    out[c] = 6 + (ip[:, 0] + 2 * ip[:, 1] + 3 * ip[:, 2]) % 4
    return out


def lower_sweep_reference(sh, N, rows, nodes, u_before, u_after, f):
    """Eq. 5.1 at each lower node from the GPU's own neighbour values at the
    state its step order implies (neighbours of an earlier step: after the
    sweep; of the same or a later step: before).  Returns the oracle's
    update and the smoother's per-node scale sum_{w != mc} |s_w x_w| + |f_I|
    divided by |s_mc|."""
    ref, scale = [], []
    for n in nodes:
        cols = np.array(list(rows[int(n)].keys()), dtype=np.int64)
        vals = np.array(list(rows[int(n)].values()))
        sn = step_of(sh, N, [int(n)])[0]
        keep = (cols != n) & ~M.dirichlet_of(sh, N, cols)
        sc = step_of(sh, N, cols[keep])
        x = np.where(sc < sn, np.asarray(u_after, dtype=np.float64)[cols[keep]],
                     np.asarray(u_before, dtype=np.float64)[cols[keep]])
        diag = vals[cols == n][0]
        acc = float(f[n]) - float(np.dot(vals[keep], x))
        ref.append(acc / diag)
        scale.append((float(np.abs(vals[keep]) @ np.abs(x)) + abs(float(f[n]))) / abs(diag))
    return np.array(ref), np.array(scale)


def cell_smoother_scale(W, lc, x, f_rows):
    """Per-node smoother scale (sum_{w != mc} |s_w x_w| + |f_I|) / |s_mc| for
    the interior rows of one cell (W: (n, 15) weights, lc: local column
    indices into x)."""
    return (np.abs(W[:, :14] * x[lc[:, :14]]).sum(axis=1) + np.abs(f_rows)) / np.abs(W[:, 14])


def assert_per_node(got, ref, scale, C, what=""):
    """max_I |got_I - ref_I| / (eps scale_I) <= C."""
    got = np.asarray(got, dtype=np.float64)
    ratio = np.abs(got - ref) / (EPS32 * np.maximum(scale, 1e-300))
    worst = float(ratio.max()) if len(ratio) else 0.0
    assert worst <= C, f"{what}: per-node error {worst:.1f} eps x scale > {C}"
    return worst
