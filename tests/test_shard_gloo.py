"""Sharding one problem over two ranks (Sec. 3.5), on the CPU with gloo.

Each rank evaluates its contiguous share of the level-s subtrees, the ranks
all-gather the subtrees' summaries (paper_1507_04789_gb300.shard), and each
finishes the coarse levels.  The evaluator here is the oracle's own two-phase
form (level-s subtrees by Eq. priorw and the posterior recursions, then the
coarse posterior from the gathered A, omega and child d, u), so the test checks
the decomposition and the orchestration: both ranks must reproduce the
single-process log-likelihood, and, through the complex step, its gradient.
"""
import math
import os
import socket

import numpy as np
import pytest

from oracle import mra_oracle as O


class OracleSubtrees:
    """The oracle behind the two-phase interface of a streamed GPU handle."""

    def __init__(self, prob, s):
        self.p, self.s = prob, s
        self.r = prob.r

    def summary_len(self):
        s, r, tree = self.s, self.r, self.p.tree
        return (s + 1) ** 2 * r * r + (s + 1) * r + 2 * O.J_at(tree.J, s + 1), tree.nreg(s)

    def loglik_subtrees(self, theta, first, count):
        p, s, tree = self.p, self.s, self.p.tree
        th, tau2 = O._split_theta(theta)
        rows = []
        for i in range(first, first + count):
            P = O.prior(tree, p.locs, th, p.family, tau2, p.nonstat, subtree=(s, i))
            Q = O.posterior(tree, p.locs, p.y, P, subtree=(s, i))
            A, om = Q.A[(s, i)], Q.omega[(s, i)]
            Jc = O.J_at(tree.J, s + 1)
            kids = [(s + 1, Jc * i + j) for j in range(Jc)]
            parts = [A[(k, l)].ravel() for k in range(s + 1) for l in range(s + 1)] + [om[k] for k in range(s + 1)]
            parts.append(np.array([v for c in kids for v in (Q.d[c], Q.u[c])]))
            rows.append(np.concatenate([np.asarray(x, dtype=np.complex128) for x in parts]))
        out = np.array(rows, dtype=np.complex128).reshape(count, self.summary_len()[0])
        return out if np.iscomplexobj(np.asarray(theta)) else out.real.copy()

    def loglik_combine(self, theta, summaries):
        p, s, r, tree = self.p, self.s, self.r, self.p.tree
        th, tau2 = O._split_theta(theta)
        P = O.prior(tree, p.locs, th, p.family, tau2, p.nonstat, levels=s)
        A_s, om_s, dk, uk = [], [], [], []
        for row in summaries:
            o = 0
            A = {}
            for k in range(s + 1):
                for l in range(s + 1):
                    A[(k, l)] = row[o:o + r * r].reshape(r, r)
                    o += r * r
            om = []
            for k in range(s + 1):
                om.append(row[o:o + r])
                o += r
            du = row[o:o + 2 * O.J_at(tree.J, s + 1)]
            A_s.append(A)
            om_s.append(om)
            dk.append(du[0::2].sum())
            uk.append(du[1::2].sum())
        Q = O.posterior_coarse(tree, P, s, A_s, om_s, dk, uk)
        n = p.locs.shape[0]
        return -0.5 * (Q.d[(0, 0)] + Q.u[(0, 0)]) - 0.5 * n * math.log(2.0 * math.pi)


def _problem(J=4):
    rng = np.random.default_rng(140)
    locs = rng.random((500, 2))
    y = rng.standard_normal(500)
    return O.Problem(locs, y, M=3, J=J, r=4, family="matern15")


THETA = np.array([1.1, 0.2, 0.06])


def _rank(rank, world, port, out_dir, J, s):
    import torch.distributed as dist

    from paper_1507_04789_gb300 import shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        ev = OracleSubtrees(_problem(J), s)
        ll = shard.sharded_loglik(ev, THETA, rank, world)
        g = []
        for a in range(3):
            tc = THETA.astype(np.complex128)
            h = 1e-30 * max(abs(THETA[a]), 1.0)
            tc[a] += 1j * h
            g.append(np.imag(shard.sharded_loglik(ev, tc, rank, world)) / h)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.array([ll, *g]))
    finally:
        dist.destroy_process_group()


def test_subtree_ranges_cover_once():
    from paper_1507_04789_gb300 import shard
    for nsub in (1, 4, 16, 17, 64):
        for world in (1, 2, 3, 8):
            got = [shard.subtree_range(nsub, k, world) for k in range(world)]
            assert sum(c for _, c in got) == nsub
            assert all(got[k][0] + got[k][1] == got[k + 1][0] for k in range(world - 1))


@pytest.mark.parametrize("J,s", [(4, 2), ((2, 8, 2), 1)])   # the quadtree; level-varying J, 8 children per subtree
def test_two_ranks_reproduce_single_process(tmp_path, J, s):
    import torch.multiprocessing as tmp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    tmp.start_processes(_rank, args=(2, port, str(tmp_path), J, s), nprocs=2, join=True, start_method="spawn")
    p = _problem(J)
    ll, g = O.loglik_grad(p, THETA)
    for k in range(2):
        v = np.load(tmp_path / f"rank{k}.npy")
        assert v[0] == pytest.approx(ll, rel=1e-12)
        np.testing.assert_allclose(v[1:], g, rtol=1e-9, atol=1e-9 * np.abs(g).max())
