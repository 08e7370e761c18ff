"""Subdomain sharding (the multi-GPU split of the subdomain batch): the exchange and
reduction logic of paper_2101_02959_gb300.shard on two CPU ranks (gloo).  The local
products each rank would compute on its GPU are stood in for by the oracle's local
Schur complements; the sharded operator, dot products and coarse right-hand side must
equal the one-rank results."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _setup(name):
    import synth
    from conftest import oracle_problem
    from oracle import ionic
    from oracle.dd import DDSolver
    from paper_2101_02959_gb300 import binding, shard
    prob = oracle_problem(name)
    ui, ue, w = synth.initial_state(prob.N, 0)
    ui = ui + 20.0 * np.exp(-np.sum(prob.mesh.coords ** 2, axis=1) / 0.02)
    wn = ionic.gating_step(ui - ue, w, prob.tau, prob.p)
    dd = DDSolver(prob)
    dd.setup(prob.p["chi_cm"] + prob.tau * ionic.di_ion_dv(ui - ue, wn, prob.p))
    pl = binding.Plan(synth.workload(name))
    sub_dofs = shard.subdomain_interface_dofs(pl.index_set("SUB_NODE_PTR"), pl.index_set("SUB_NODES"),
                                              pl.index_set("SUB_NINT"), pl.index_set("IFACE_NODES"))
    return prob, dd, sub_dofs


def _rank(rank, world, port, name, out):
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2101_02959_gb300 import shard
        prob, dd, sub_dofs = _setup(name)
        n = prob.dofs.n_iface
        plan = shard.ShardPlan(sub_dofs, n, world, rank)
        rng = np.random.default_rng(3)
        x = rng.standard_normal(n)
        y = rng.standard_normal(n)
        # this rank's local products S^(j) R_j x, summed onto the interface (R_j^T)
        partial = np.zeros(n)
        for j in plan.subs:
            L = dd.loc[j]
            np.add.at(partial, L["R"], L["S"] @ x[L["R"]])
        got = plan.assemble(torch.from_numpy(partial)).numpy()
        # coarse right-hand side: this rank's local primal contributions Phi_D^(j)T r_D
        cr = np.zeros(prob.part.n_primal)
        for j in plan.subs:
            L = dd.loc[j]
            np.add.at(cr, L["primal"], L["PhiD"].T @ np.ones(len(L["dual"])))
        cr_all = plan.allreduce(torch.from_numpy(cr)).numpy()
        out[rank] = dict(touched=plan.touched, assembled=got[plan.touched],
                         dot=plan.dot(torch.from_numpy(x), torch.from_numpy(y)), coarse=cr_all, subs=plan.subs,
                         shared=dict(plan.shared))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("name,world", [("cube8ve", 2), ("ragged", 2), ("cube8ve", 3)])
def test_sharded_operator_matches_one_rank(name, world):
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_rank, args=(world, port, name, out), nprocs=world, join=True)
    prob, dd, sub_dofs = _setup(name)
    # the plan's interface dofs of every subdomain are the oracle's R_j
    for j, L in enumerate(dd.loc):
        np.testing.assert_array_equal(sub_dofs[j], L["R"])
    n = prob.dofs.n_iface
    rng = np.random.default_rng(3)
    x = rng.standard_normal(n)
    y = rng.standard_normal(n)
    ref = dd.schur_apply(x)  # one rank: S_hat x (gauge dof zeroed)
    g = dd.g_iface
    subs = np.concatenate([out[r]["subs"] for r in range(world)])
    assert sorted(subs.tolist()) == list(range(prob.part.n_sub))
    assert all(len(out[r]["subs"]) > 0 for r in range(world)) and out[0]["shared"]
    for r in range(world):
        t, a = out[r]["touched"], out[r]["assembled"]
        keep = t != g
        np.testing.assert_allclose(a[keep], ref[t[keep]], rtol=0, atol=1e-13 * np.abs(ref).max())
        assert abs(out[r]["dot"] - x @ y) <= 1e-12 * np.abs(x) @ np.abs(y)
    # a dof shared by two ranks has the same value, bit for bit, on both
    pairs = 0
    for ra in range(world):
        for rb in range(ra + 1, world):
            ta, aa = out[ra]["touched"], out[ra]["assembled"]
            tb, ab = out[rb]["touched"], out[rb]["assembled"]
            common, ia, ib = np.intersect1d(ta, tb, return_indices=True)
            pairs += common.size > 0
            np.testing.assert_array_equal(aa[ia], ab[ib])
    assert pairs > 0
    # coarse right-hand side: the sum over all subdomains, replicated
    full = np.zeros(prob.part.n_primal)
    for L in dd.loc:
        np.add.at(full, L["primal"], L["PhiD"].T @ np.ones(len(L["dual"])))
    for r in range(world):
        np.testing.assert_allclose(out[r]["coarse"], full, rtol=1e-13, atol=1e-13 * np.abs(full).max())


def test_block_partition():
    from paper_2101_02959_gb300 import shard
    p = shard.block_partition(10, 3)
    assert p.tolist() == [0, 0, 0, 0, 1, 1, 1, 2, 2, 2]
    assert shard.block_partition(4, 1).tolist() == [0, 0, 0, 0]
