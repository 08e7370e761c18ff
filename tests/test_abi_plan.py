"""C-ABI without a GPU: the library loads, exports what include/bidomain.h
declares, and its host-built index sets equal the oracle's bit for bit."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from conftest import ROOT, oracle_problem
from paper_2101_02959_gb300 import binding, build


@pytest.fixture(scope="module")
def lib():
    build.build()
    return binding.load()


def test_exports_every_declared_symbol(lib):
    hdr = open(os.path.join(ROOT, "include", "bidomain.h")).read()
    names = set(re.findall(r"^(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", hdr, flags=re.M))
    assert len(names) >= 20
    assert names == set(binding.EXPORTED)
    for n in names:
        assert hasattr(lib, n), n


def test_strerror_and_bad_args(lib):
    assert lib.bidomain_strerror(0) == b"ok"
    assert b"positive" in lib.bidomain_strerror(-2)
    w = synth.workload("cube8")
    bad = dict(w, s=(0, 4, 4))
    with pytest.raises(binding.BidomainError):
        binding.Plan(bad)
    # one subdomain: no interface, so no vertex to hold the gauge
    with pytest.raises(binding.BidomainError):
        binding.Plan(dict(w, s=(8, 8, 8)))
    # ellipsoid ranges must avoid the poles and have positive axes
    e = synth.workload("ell8")
    for bad in (dict(e["ellipsoid"], theta=(-1.0, 1.6)), dict(e["ellipsoid"], phi=(0.5, 0.0)),
                dict(e["ellipsoid"], axes=(1.5, 2.7, 0.0, 2.7, 4.4, 5.0))):
        with pytest.raises(binding.BidomainError):
            binding.Plan(dict(e, ellipsoid=bad))
    binding.Plan(e)


def _oracle_sets(prob):
    p, d = prob.part, prob.dofs
    out = {
        "ELEM_SUB": p.elem_sub,
        "NODE_MULT": p.mult,
        "IFACE_NODES": p.iface_nodes,
        "CLS_TYPE": p.cls_type,
        "CLS_PTR": np.concatenate([[0], np.cumsum([len(c) for c in p.cls_nodes])]),
        "CLS_NODES": np.concatenate(p.cls_nodes),
        "CLS_SUB_PTR": np.concatenate([[0], np.cumsum([len(c) for c in p.cls_subs])]),
        "CLS_SUBS": np.concatenate([np.array(c) for c in p.cls_subs]),
        "CLS_DUAL_START": d.cls_dual_start,
        "GAUGE": np.array([p.gauge_node, p.gauge_primal]),
    }
    nodes, nint, dual, primal = [], [], [], []
    for j in range(p.n_sub):
        L = d.local(j)
        nodes.append(np.concatenate([L["interior_nodes"], L["iface_nodes"]]))
        nint.append(len(L["interior_nodes"]))
        dual.append(L["dual"])
        primal.append(L["primal"])
    out["SUB_NODES"] = np.concatenate(nodes)
    out["SUB_NINT"] = np.array(nint)
    out["SUB_DUAL"] = np.concatenate(dual)
    out["SUB_PRIMAL"] = np.concatenate(primal)
    out["SUB_DUAL_PTR"] = np.concatenate([[0], np.cumsum([len(x) for x in dual])])
    out["SUB_PRIMAL_PTR"] = np.concatenate([[0], np.cumsum([len(x) for x in primal])])
    return out


@pytest.mark.parametrize("name", ["tiny", "cube8", "cube8ve", "cube8vef", "ragged", "opt4", "ell8", "ell10",
                                  "coarse2k", "shell_small"])
def test_index_sets_bit_exact(lib, name):
    prob = oracle_problem(name)
    plan = binding.Plan(prob.workload)
    ref = _oracle_sets(prob)
    for k, v in ref.items():
        got = plan.index_set(k)
        assert got.dtype == np.int64
        np.testing.assert_array_equal(got, np.asarray(v, np.int64), err_msg=k)
    sz = plan.sizes()
    assert sz["n_node"] == prob.N
    assert sz["n_iface"] == prob.dofs.n_iface
    assert sz["n_dual"] == prob.dofs.n_dual
    assert sz["n_primal"] == prob.part.n_primal


def test_slab32_sizes(lib):
    plan = binding.Plan(synth.workload("slab32"))
    sz = plan.sizes()
    assert sz["n_node"] == 33 * 33 * 17
    assert sz["n_sub"] == 32
    assert sz["n_primal"] == 102
    t = plan.index_set("CLS_TYPE")
    assert [int((t == k).sum()) for k in range(3)] == [9, 42, 64]


@pytest.mark.parametrize("bad", [dict(method="fetidp", precond_every=2), dict(precond_every=0),
                                 dict(scaling=7)])
def test_setup_rejects_bad_options_before_touching_the_device(lib, bad):
    """Option checks run before any CUDA call, so they hold on a machine without a GPU."""
    w = synth.workload("cube8ve")
    with pytest.raises(binding.BidomainError) as e:
        binding.Solver(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, **bad)
    assert binding.ERRORS[e.value.code] == "BD_ERR_ARG"


def test_vertexless_split_promotes_a_vertex(lib):
    """Two subdomains side by side (2x1x1 blocks of the 8^3 cube) share only a face: the
    first subdomain has no vertex, so the lowest-id node of that face (grid node (4,0,0),
    id 4) becomes a vertex and the other 80 nodes of the x = 4 plane stay a face; the
    oracle applies the same rule."""
    w = dict(synth.workload("cube8"), s=(4, 8, 8), primal="VE")
    plan = binding.Plan(w)
    assert plan.index_set("CLS_TYPE").tolist() == [0, 2]
    assert plan.index_set("CLS_PTR").tolist() == [0, 1, 81]
    nodes = plan.index_set("CLS_NODES")
    assert nodes[0] == 4 and sorted(nodes[1:]) == sorted(x + 9 * y + 81 * z for z in range(9) for y in range(9)
                                                          for x in (4,) if (y, z) != (0, 0))
    assert plan.sizes()["n_primal"] == 2 and plan.index_set("GAUGE").tolist() == [4, 1]
    from oracle.bidomain import Problem
    prob = Problem(w, synth.SIGMA_I, synth.SIGMA_E, synth.IONIC, synth.TAU, synth.stimulus(w))
    ref = _oracle_sets(prob)
    for k, v in ref.items():
        np.testing.assert_array_equal(plan.index_set(k), np.asarray(v, np.int64), err_msg=k)
