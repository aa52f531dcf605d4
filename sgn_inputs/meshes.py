"""Structured meshes and seeded problem instances.

Workload shapes follow the paper's inverse elastic design example (Sec. 5,
"Inverse Elastic Design"): an elastic body clamped on one side, loaded, whose
equilibrium is pulled towards a target shape by per-element material
parameters.  The paper's own meshes are not available; these generators stand
in for them with structured triangle / tetrahedron grids.

Only geometry, connectivity, boundary conditions, loads, targets and random
draws live here.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import permutations

import numpy as np


def grid2d(n: int):
    """n x n nodes on [0,1]^2; every grid square is split along its
    (i,j)->(i+1,j+1) diagonal into two counter-clockwise triangles.

    Returns X (n*n, 2) float64 and tri (2*(n-1)^2, 3) int32.  Node (i, j)
    (i along x, j along y) has index j*n + i.
    """
    if n < 2:
        raise ValueError("grid2d needs n >= 2")
    h = 1.0 / (n - 1)
    jj, ii = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    X = np.stack([ii.ravel() * h, jj.ravel() * h], axis=1).astype(np.float64)
    i, j = np.meshgrid(np.arange(n - 1), np.arange(n - 1), indexing="ij")
    i = i.ravel(); j = j.ravel()
    v00 = j * n + i
    v10 = j * n + i + 1
    v01 = (j + 1) * n + i
    v11 = (j + 1) * n + i + 1
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    tri = np.empty((2 * len(v00), 3), dtype=np.int32)
    tri[0::2] = t1
    tri[1::2] = t2
    return X, tri


def kuhn3d(n: int):
    """n^3 nodes on [0,1]^3; every cube is split into the six tetrahedra of
    the Kuhn (Freudenthal) triangulation around its (0,0,0)->(1,1,1)
    diagonal, the same split in every cube, so the mesh is conforming and
    every interior node has 14 neighbours.  All tets are positively oriented.

    Returns X (n^3, 3) float64 and tet (6*(n-1)^3, 4) int32.  Node (i,j,k)
    has index (k*n + j)*n + i.
    """
    if n < 2:
        raise ValueError("kuhn3d needs n >= 2")
    h = 1.0 / (n - 1)
    kk, jj, ii = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    X = np.stack([ii.ravel() * h, jj.ravel() * h, kk.ravel() * h], axis=1).astype(np.float64)
    k, j, i = np.meshgrid(np.arange(n - 1), np.arange(n - 1), np.arange(n - 1), indexing="ij")
    base = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)  # cube corner
    unit = np.eye(3, dtype=np.int64)
    tets = []
    for perm in permutations(range(3)):
        c0 = base
        c1 = c0 + unit[perm[0]]
        c2 = c1 + unit[perm[1]]
        c3 = c2 + unit[perm[2]]
        # orientation sign of the path e_p0, e_p1, e_p2 is the permutation parity
        inv = sum(1 for a in range(3) for b in range(a + 1, 3) if perm[a] > perm[b])
        verts = [c0, c1, c2, c3] if inv % 2 == 0 else [c0, c2, c1, c3]
        idx = [(v[:, 2] * n + v[:, 1]) * n + v[:, 0] for v in verts]
        tets.append(np.stack(idx, axis=1))
    tet = np.stack(tets, axis=1).reshape(-1, 4).astype(np.int32)
    return X, tet


@dataclass
class Problem:
    """One equilibrium-constrained design instance.

    dim         2 or 3
    X           rest positions, (n_nodes, dim) float64
    conn        element connectivity, (n_elem, dim+1) int32
    fixed_node  1 where the node is Dirichlet-fixed (all its DOFs), uint8
    fext        external nodal force, (n_nodes, dim) float64
    track_dof   global DOF ids node*dim+comp of the tracked coordinates
    target      target value of each tracked coordinate
    weight      weight of each tracked coordinate (objective 1/2 sum w r^2)
    alpha       Tikhonov weight on p (objective alpha/2 ||p||^2)
    E0, nu      reference Young's modulus and Poisson ratio
    p0          design vector: per-element log-modulus, E_e = E0 exp(p_e)
    """
    name: str
    dim: int
    X: np.ndarray
    conn: np.ndarray
    fixed_node: np.ndarray
    fext: np.ndarray
    track_dof: np.ndarray
    target: np.ndarray
    weight: np.ndarray
    alpha: float
    E0: float
    nu: float
    p0: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self) -> int:
        return self.X.shape[0]

    @property
    def n_elem(self) -> int:
        return self.conn.shape[0]

    @property
    def n_free(self) -> int:
        return int(np.count_nonzero(self.fixed_node == 0))


def _lumped_body_load_2d(X, tri, load_per_area):
    """Body load (0, -load_per_area) per unit area, lumped equally (area/3)
    onto the three vertices of each triangle."""
    a = X[tri[:, 1]] - X[tri[:, 0]]
    b = X[tri[:, 2]] - X[tri[:, 0]]
    area = 0.5 * np.abs(a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0])
    f = np.zeros_like(X)
    for v in range(3):
        np.add.at(f[:, 1], tri[:, v], -load_per_area * area / 3.0)
    return f


def problem_2d(n: int = 21, seed: int = 0, E0: float = 1e4, nu: float = 0.3,
               body_load: float = 10.0, shift=(0.0, -0.05), alpha: float = 1e-4,
               p_sigma: float = 0.1, name: str | None = None) -> Problem:
    """Plane-strain bar on the unit square: left edge clamped, uniform
    downward body load, right-edge nodes tracked towards their rest position
    shifted by `shift`; p drawn i.i.d. N(0, p_sigma^2) with `seed`."""
    X, tri = grid2d(n)
    fixed = (np.abs(X[:, 0]) < 1e-12).astype(np.uint8)
    fext = _lumped_body_load_2d(X, tri, body_load)
    right = np.nonzero(np.abs(X[:, 0] - 1.0) < 1e-12)[0]
    track_dof = np.stack([right * 2, right * 2 + 1], axis=1).ravel().astype(np.int64)
    target = (X[right] + np.asarray(shift, dtype=np.float64)[None, :]).ravel()
    rng = np.random.default_rng(seed)
    p0 = rng.normal(0.0, p_sigma, size=tri.shape[0]) if p_sigma > 0 else np.zeros(tri.shape[0])
    return Problem(name or f"grid2d_{n}", 2, X, tri, fixed, fext, track_dof, target,
                   np.ones(track_dof.shape[0]), alpha, E0, nu, p0.astype(np.float64),
                   meta={"n": n, "seed": seed})


def _smooth_target_height(XY, rng, n_waves=8, amplitude=0.02):
    """Sum of `n_waves` sinusoids sin(2 pi (a X + b Y) + phi), a, b ~ U{1,2,3},
    phi ~ U[0, 2 pi), scaled to max |.| = amplitude on the given points."""
    a = rng.integers(1, 4, size=n_waves)
    b = rng.integers(1, 4, size=n_waves)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n_waves)
    h = np.zeros(XY.shape[0])
    for k in range(n_waves):
        h += np.sin(2.0 * np.pi * (a[k] * XY[:, 0] + b[k] * XY[:, 1]) + phi[k])
    return amplitude * h / np.max(np.abs(h))


def problem_3d(n: int = 40, seed: int = 0, E0: float = 1e4, nu: float = 0.3,
               alpha: float = 1e-4, p_sigma: float = 0.0, load_scale: float = 1.0,
               name: str | None = None) -> Problem:
    """Kuhn-tet cube: bottom face (z=0) clamped, top-face nodes loaded by
    -z * u_i * load_scale with u_i ~ U[0,1]; all three coordinates of the
    top-face nodes tracked towards rest + (0, 0, g(X, Y)) with g a seeded
    sum of 8 sinusoids of amplitude 0.02; p = 0 unless p_sigma > 0."""
    X, tet = kuhn3d(n)
    rng = np.random.default_rng(seed)
    fixed = (np.abs(X[:, 2]) < 1e-12).astype(np.uint8)
    top = np.nonzero(np.abs(X[:, 2] - 1.0) < 1e-12)[0]
    fext = np.zeros_like(X)
    fext[top, 2] = -load_scale * rng.uniform(0.0, 1.0, size=top.shape[0])
    g = _smooth_target_height(X[top, :2], rng)
    target = X[top].copy()
    target[:, 2] += g
    track_dof = np.stack([top * 3, top * 3 + 1, top * 3 + 2], axis=1).ravel().astype(np.int64)
    p0 = rng.normal(0.0, p_sigma, size=tet.shape[0]) if p_sigma > 0 else np.zeros(tet.shape[0])
    return Problem(name or f"kuhn3d_{n}", 3, X, tet, fixed, fext, track_dof, target.ravel(),
                   np.ones(track_dof.shape[0]), alpha, E0, nu, p0.astype(np.float64),
                   meta={"n": n, "seed": seed})


def problem_tiny_2d(n: int = 4, seed: int = 1, p_sigma: float = 0.2) -> Problem:
    """A few-element 2D instance for finite-difference and brute-force pins."""
    return problem_2d(n=n, seed=seed, p_sigma=p_sigma, name=f"tiny2d_{n}")


def problem_tiny_3d(n: int = 3, seed: int = 1, p_sigma: float = 0.2) -> Problem:
    """A few-element 3D instance for finite-difference and brute-force pins."""
    return problem_3d(n=n, seed=seed, p_sigma=p_sigma, name=f"tiny3d_{n}")


def batch2d_instances(n_instances: int = 256, seed: int = 0, side_lo: int = 10, side_hi: int = 60,
                      shift_sigma: float = 0.03, p_sigma: float = 0.1) -> list:
    """Many independent plane-strain design instances of uneven size.

    Instance i is a side_i x side_i grid on the unit square (side_i ~
    U{side_lo..side_hi}), clamped on its left edge, body-loaded, with its right
    edge tracked towards rest + (0, -0.05) + s_i where s_i ~ N(0, shift_sigma^2)
    (one 2-vector per instance); p ~ N(0, p_sigma^2).  Every instance keeps its
    own coordinates."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=n_instances)
    out = []
    for n in sides:
        shift = (0.0, -0.05) + rng.normal(0.0, shift_sigma, size=2)
        sub = problem_2d(int(n), seed=int(rng.integers(0, 2**31 - 1)), shift=tuple(shift), p_sigma=p_sigma)
        out.append(sub)
    return out


def problem_batch2d(n_instances: int = 256, seed: int = 0, side_lo: int = 10, side_hi: int = 60,
                    shift_sigma: float = 0.03, p_sigma: float = 0.1, gap: float = 0.5) -> Problem:
    """The instances of batch2d_instances joined into one disjoint mesh by
    hand: they sit on a square grid of cells (1 + gap) apart, so they never
    share nodes; meta["node_offsets"] and meta["elem_offsets"] delimit them,
    meta["origins"] holds each instance's translation."""
    subs = batch2d_instances(n_instances, seed, side_lo, side_hi, shift_sigma, p_sigma)
    sides = np.array([int(round(np.sqrt(sub.n_nodes))) for sub in subs])
    Xs, conns, fixeds, fexts, tracks, targets, weights, ps = [], [], [], [], [], [], [], []
    node_off, elem_off = [0], [0]
    per_row = int(np.ceil(np.sqrt(n_instances)))
    origins = np.array([((i % per_row) * (1.0 + gap), (i // per_row) * (1.0 + gap)) for i in range(n_instances)])
    for i, sub in enumerate(subs):
        X = sub.X + origins[i]
        tgt = sub.target.reshape(-1, 2) + origins[i]
        Xs.append(X)
        conns.append(sub.conn + node_off[-1])
        fixeds.append(sub.fixed_node)
        fexts.append(sub.fext)
        tracks.append(sub.track_dof + 2 * node_off[-1])
        targets.append(tgt.ravel())
        weights.append(sub.weight)
        ps.append(sub.p0)
        node_off.append(node_off[-1] + X.shape[0])
        elem_off.append(elem_off[-1] + sub.conn.shape[0])
    return Problem(f"batch2d_{n_instances}", 2, np.concatenate(Xs), np.concatenate(conns).astype(np.int32),
                   np.concatenate(fixeds), np.concatenate(fexts), np.concatenate(tracks),
                   np.concatenate(targets), np.concatenate(weights), 1e-4, 1e4, 0.3, np.concatenate(ps),
                   meta={"sides": sides, "node_offsets": np.array(node_off), "elem_offsets": np.array(elem_off),
                         "seed": seed, "side_lo": side_lo, "side_hi": side_hi, "shift_sigma": shift_sigma,
                         "p_sigma": p_sigma, "origins": origins})


def select_instances(batch: Problem, idx) -> Problem:
    """The sub-batch of problem_batch2d's instances idx (in that order), with
    their own node / element numbering, loads, targets and parameters."""
    no, eo = batch.meta["node_offsets"], batch.meta["elem_offsets"]
    idx = [int(i) for i in idx]
    node_map = -np.ones(batch.n_nodes, dtype=np.int64)
    nodes, elems, node_off, elem_off = [], [], [0], [0]
    for i in idx:
        nn = np.arange(no[i], no[i + 1])
        node_map[nn] = node_off[-1] + np.arange(nn.size)
        nodes.append(nn)
        elems.append(np.arange(eo[i], eo[i + 1]))
        node_off.append(node_off[-1] + nn.size)
        elem_off.append(elem_off[-1] + eo[i + 1] - eo[i])
    nodes = np.concatenate(nodes)
    elems = np.concatenate(elems)
    tr = batch.track_dof.reshape(-1)
    keep = np.isin(tr // 2, nodes)
    track = node_map[tr[keep] // 2] * 2 + tr[keep] % 2
    order = np.argsort(track, kind="stable")
    target = batch.target.reshape(-1)[keep]
    weight = batch.weight.reshape(-1)[keep]
    meta = dict(batch.meta)
    meta.update({"sides": np.asarray(batch.meta["sides"])[idx], "node_offsets": np.array(node_off),
                 "elem_offsets": np.array(elem_off), "origins": np.asarray(batch.meta["origins"])[idx],
                 "instances": np.array(idx)})
    return Problem(f"{batch.name}_sel{len(idx)}", 2, batch.X[nodes], node_map[batch.conn[elems]].astype(np.int32),
                   batch.fixed_node[nodes], batch.fext[nodes], track[order].astype(np.int64), target[order],
                   weight[order], batch.alpha, batch.E0, batch.nu, batch.p0[elems], meta=meta)


def problem_rbf3d(n: int = 40, n_rbf: int = 64, width: float = 0.15, seed: int = 0,
                  theta_sigma: float = 0.3, load_scale: float | None = None) -> Problem:
    """The 3D cube of problem_3d whose per-tet log-modulus field is given by
    n_rbf Gaussian radial basis functions: p_e = sum_k theta_k
    exp(-|X_e - c_k|^2 / (2 width^2)) at the tet centroid X_e, with centres
    c_k ~ U[0,1]^3 (seeded).  meta holds the centres, the width and theta_sigma
    (coefficient vectors theta ~ N(0, theta_sigma^2), see draw_thetas).
    load_scale defaults to (40 / n)^2 (n nodes per side): every resolution
    carries the total top-face load of the 40^3-node cube (about 15% peak
    displacement, four to five Newton iterations from the rest shape)."""
    if load_scale is None:
        load_scale = (40.0 / n) ** 2
    prob = problem_3d(n, seed=seed, load_scale=load_scale)
    rng = np.random.default_rng(seed + 7919)
    centers = rng.uniform(0.0, 1.0, size=(n_rbf, 3))
    prob.name = f"rbf3d_{n}"
    prob.meta.update({"rbf_centers": centers, "rbf_width": width, "theta_sigma": theta_sigma,
                      "n_rbf": n_rbf})
    return prob


def draw_thetas(prob: Problem, count: int, seed: int) -> np.ndarray:
    """count coefficient vectors theta ~ N(0, theta_sigma^2) for an RBF problem."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, prob.meta["theta_sigma"], size=(count, prob.meta["n_rbf"]))


PRESETS = {
    # 21x21 plane-strain grid, 800 triangles, p ~ N(0, 0.1^2)
    "grid2d_21": lambda seed=0: problem_2d(21, seed=seed),
    # 40^3 Kuhn tets, 355,914 elements, p = 0
    "kuhn3d_40": lambda seed=0: problem_3d(40, seed=seed),
    # 80^3 Kuhn tets, 2,958,234 elements; the same cube under the same total
    # top-face load as kuhn3d_40 (per-node loads scaled by (40/80)^2)
    "kuhn3d_80": lambda seed=0: problem_3d(80, seed=seed, load_scale=0.25, name="kuhn3d_80"),
    # 40^3 cube with 64 RBF design coefficients (learned warm start)
    "rbf3d_40": lambda seed=0: problem_rbf3d(40, seed=seed),
    # 256 plane-strain instances, sides ~ U{10..60}
    "batch2d_256": lambda seed=0: problem_batch2d(256, seed=seed),
}


def make_preset(name: str, seed: int = 0) -> Problem:
    if name in PRESETS:
        return PRESETS[name](seed)
    # "kuhn3d_<n>" / "grid2d_<n>" for any n
    kind, _, size = name.rpartition("_")
    if kind == "kuhn3d":
        return problem_3d(int(size), seed=seed)
    if kind == "grid2d":
        return problem_2d(int(size), seed=seed)
    if kind == "batch2d":
        return problem_batch2d(int(size), seed=seed)
    if kind == "rbf3d":
        return problem_rbf3d(int(size), seed=seed)
    raise KeyError(name)
