"""The row-block partition plan (pfc_host_partition) and a partitioned stage solve on CPU ranks.

The paper runs its solver on MPI processes that own contiguous row blocks, with a
halo exchange per matrix-vector product and a global sum per inner product
(Section 7).  A multi-device solve here would use the library's strip plan; no run
of this build has more than one GPU, so the partitioned algorithm is exercised as
`gloo` ranks on the CPU: FGMRES(30) with modified Gram-Schmidt around P_CH with
Jacobi-PCG inner solves (Section 4, Table 2), every product after a ghost exchange
with the two neighbouring ranks only (the plan's halo), every inner product an
all-reduce.  The gathered solution must match a sparse direct solve of the
oracle's stage system to 1e-8; the plan itself is checked against the pattern."""
import math
import os
import socket

import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synth
from oracle.mesh import structured_mesh
from oracle.rosenbrock import ROS3PW, PFCProblem

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import paper_1501_06852_gb300 as pfc  # noqa: E402

CASE = (2, 12, 6.0, -0.4, -0.3, 0.1)   # 2D, h = 0.5 (the spacing of the 512^2 workload), 625 dofs/field
TAU = 1.0


@pytest.mark.parametrize("dim,side,L,nparts,degree", [(2, 12, 6.0, 2, 2), (2, 512, 256.0, 4, 2),
                                                      (3, 8, 8.0, 3, 2), (2, 12, 6.0, 5, 1)])
def test_plan_covers_every_column_and_balances(dim, side, L, nparts, degree):
    plan = pfc.host_partition(dim, side, L, nparts, degree)
    lat = degree * side + 1
    n = lat ** dim
    line = lat ** (dim - 1)
    b = plan["begin"]
    assert b[0] == 0 and b[-1] == n and all(x % line == 0 for x in b)
    assert all(b[k + 1] - b[k] >= degree * line for k in range(nparts))
    hp = pfc.host_pattern(dim, side, L)
    if degree == 2:
        assert sum(plan["nnz"]) == hp["nnz"]
    if side <= 16:
        prob = PFCProblem(structured_mesh(dim, side, L, degree=degree), -0.4)
        M = prob.M.tocsr()
        for k in range(nparts):
            rows = M[b[k]:b[k + 1]]
            lo, hi = rows.indices.min(), rows.indices.max()
            below, above = plan["halo"][k]
            assert lo == b[k] - below and hi == b[k + 1] + above - 1
            assert rows.nnz == plan["nnz"][k]
    mean = sum(plan["nnz"]) / nparts
    assert max(plan["nnz"]) <= 1.25 * mean


def test_plan_rejects_too_many_parts():
    with pytest.raises(pfc.PFCError):
        pfc.host_partition(2, 4, 4.0, 5)          # 9 lattice lines, 2 per part at least


# ----------------------------------------------------------------------------- partitioned solve
class Part:
    """This rank's rows of every field and its ghost exchange with the neighbours."""

    def __init__(self, plan, rank, world, n):
        self.rank, self.world, self.n = rank, world, n
        self.lo, self.hi = plan["begin"][rank], plan["begin"][rank + 1]
        self.halo = plan["halo"]

    def own(self, nf):
        return np.concatenate([np.arange(f * self.n + self.lo, f * self.n + self.hi) for f in range(nf)])

    def full(self, v_own, nf):
        """Full-length vector with this rank's rows and its ghost rows filled."""
        n, lo, hi, m = self.n, self.lo, self.hi, self.hi - self.lo
        out = np.zeros(nf * n)
        reqs, recv = [], []
        for f in range(nf):
            out[f * n + lo:f * n + hi] = v_own[f * m:(f + 1) * m]
            if self.rank > 0:       # my lowest rows are the lower neighbour's upper ghosts
                k = self.halo[self.rank - 1][1]
                reqs.append(dist.isend(torch.from_numpy(out[f * n + lo:f * n + lo + k].copy()), self.rank - 1, tag=f))
                k = self.halo[self.rank][0]
                buf = torch.empty(k, dtype=torch.float64)
                reqs.append(dist.irecv(buf, self.rank - 1, tag=10 + f))
                recv.append((f * n + lo - k, buf))
            if self.rank + 1 < self.world:
                k = self.halo[self.rank + 1][0]
                reqs.append(dist.isend(torch.from_numpy(out[f * n + hi - k:f * n + hi].copy()), self.rank + 1,
                                       tag=10 + f))
                k = self.halo[self.rank][1]
                buf = torch.empty(k, dtype=torch.float64)
                reqs.append(dist.irecv(buf, self.rank + 1, tag=f))
                recv.append((f * n + hi, buf))
        for r in reqs:
            r.wait()
        for start, buf in recv:
            out[start:start + buf.numel()] = buf.numpy()
        return out


def _dot(a, b):
    t = torch.tensor([float(a @ b)], dtype=torch.float64)
    dist.all_reduce(t)
    return float(t.item())


def _pcg(part, A_rows, dinv, rhs, rtol=1e-3, maxit=10000):
    """Jacobi-PCG from zero on this rank's rows (Table 2)."""
    x = np.zeros_like(rhs)
    bb = math.sqrt(_dot(rhs, rhs))
    if bb == 0.0:
        return x
    r = rhs.copy()
    z = dinv * r
    p = z.copy()
    rz = _dot(r, z)
    for _ in range(maxit):
        q = A_rows @ part.full(p, 1)
        alpha = rz / _dot(p, q)
        x += alpha * p
        r -= alpha * q
        if math.sqrt(_dot(r, r)) <= rtol * bb:
            break
        z = dinv * r
        rz_new = _dot(r, z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


def _rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dim, side, L, r, pm, amp = CASE
        prob = PFCProblem(structured_mesh(dim, side, L), r)
        n = prob.n
        x0 = prob.consistent_state(synth.initial_psi(dim, side, pm, amp, 2))
        A = prob.stage_matrix(x0[n:2 * n], TAU).tocsr()
        b = prob.stage_rhs(x0, [], [], TAU)
        plan = pfc.host_partition(dim, side, L, world)
        part = Part(plan, rank, world, n)
        own1, own3 = part.own(1), part.own(3)
        A_rows = A[own3]
        gamma = ROS3PW.gamma
        tau_e = gamma * TAU
        delta = math.sqrt(tau_e)
        M, K = prob.M.tocsr(), prob.K.tocsr()
        mats = {"M": M, "K": K, "MdK": (M + delta * K).tocsr(), "MsK": (M + math.sqrt(delta) * K).tocsr()}
        rows = {k: v[own1] for k, v in mats.items()}
        dinv = {k: 1.0 / mats[k].diagonal()[own1] for k in ("M", "MdK", "MsK")}
        m = own1.size

        def pch(v):          # steps (1)-(5) of P_CH on this rank's rows
            v0, v1, v2 = v[:m], v[m:2 * m], v[2 * m:]
            y0 = _pcg(part, rows["M"], dinv["M"], v0)
            y1 = _pcg(part, rows["MdK"], dinv["MdK"], gamma * v1 - tau_e * (rows["K"] @ part.full(y0, 1)))
            w = _pcg(part, rows["MsK"], dinv["MsK"], rows["M"] @ part.full(y1, 1))
            x1 = _pcg(part, rows["MsK"], dinv["MsK"], rows["M"] @ part.full(w, 1))
            xx0 = y0 + (y1 - x1) / delta
            x2 = _pcg(part, rows["M"], dinv["M"], v2 - rows["K"] @ part.full(x1, 1))
            return np.concatenate([xx0, x1, x2])

        def apply_A(v):
            return A_rows @ part.full(v, 3)

        # FGMRES(30) + MGS, zero start, true residual at each restart (Section 4, 7)
        bl = b[own3]
        y = np.zeros_like(bl)
        bn = math.sqrt(_dot(bl, bl))
        tol, restart = 1e-12, 30
        while True:
            res = bl - apply_A(y)
            beta = math.sqrt(_dot(res, res))
            if beta <= tol * bn:
                break
            V, Z = [res / beta], []
            H = np.zeros((restart + 1, restart))
            g = np.zeros(restart + 1)
            g[0] = beta
            k = 0
            for j in range(restart):
                z = pch(V[j])
                Z.append(z)
                w = apply_A(z)
                for i in range(j + 1):
                    H[i, j] = _dot(w, V[i])
                    w = w - H[i, j] * V[i]
                H[j + 1, j] = math.sqrt(_dot(w, w))
                k = j + 1
                c, *_ = np.linalg.lstsq(H[:j + 2, :j + 1], g[:j + 2], rcond=None)
                if np.linalg.norm(g[:j + 2] - H[:j + 2, :j + 1] @ c) <= tol * bn:
                    break
                V.append(w / H[j + 1, j])
            y = y + np.array(Z[:k]).T @ c
        parts = [None] * world
        dist.all_gather_object(parts, (own3.tolist(), y.tolist()))
        if rank == 0:
            full = np.zeros(3 * n)
            for idx, vals in parts:
                full[np.array(idx)] = vals
            np.save(out_path, full)
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 3])
def test_partitioned_stage_solve_matches_direct_solve(world, tmp_path):
    out = str(tmp_path / "y.npy")
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    dim, side, L, r, pm, amp = CASE
    prob = PFCProblem(structured_mesh(dim, side, L), r)
    n = prob.n
    x0 = prob.consistent_state(synth.initial_psi(dim, side, pm, amp, 2))
    A = prob.stage_matrix(x0[n:2 * n], TAU)
    b = prob.stage_rhs(x0, [], [], TAU)
    y_ex = spla.splu(A.tocsc()).solve(b)
    y = np.load(out)
    assert np.linalg.norm(y - y_ex) <= 1e-8 * np.linalg.norm(y_ex)
