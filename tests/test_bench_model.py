"""The bench's algorithmic work model and roofline arithmetic (host code of bench.py): the
per-subdomain flop and byte counts follow their closed forms, the Krylov figure takes the lesser
of the banded factors and the packed explicit operators, uneven workloads are capped at what the
launches do, and a traffic figure is dropped once the kernel source no longer matches."""
import numpy as np
import pytest

import bench


def test_local_shapes_and_factor_flops_at_hh8():
    pd, md, pn, mn, ng, ni, nf = bench.local_shapes(8)
    assert (pd, md, pn, mn) == (7, 98, 9, 162)
    assert ng == 2 * (9 ** 3 - 7 ** 3) == 772 and ni == 686 and nf == 98
    fd, fn = 1.5 * pd * md ** 2, 1.5 * pn * mn ** 2
    want = 2.33 * pd * md ** 3 + 2.33 * pn * mn ** 3 + 2.0 * fd * ng + ni * 6 * nf ** 2 + 4.0 * fn * 40
    assert bench.factor_flops_per_sub(8) == pytest.approx(want, rel=1e-15)
    assert bench.factor_flops_per_sub(8) == pytest.approx(3.56e8, rel=0.01)


def test_explicit_values_are_packed_triangles():
    assert bench.explicit_values_per_sub(772, 730, 42) == 772 * 773 / 2 + 730 * 731 / 2 + 42 * 730
    vd, vn = bench.solve_values_per_sub(8)
    assert bench.explicit_values_per_sub(772, 730, 42) < vd + vn  # fewer bytes than the banded solves


def _prof(gemv_bytes):
    return {"panel": {"ms": 150.0, "launches": 900, "flops": 2e12, "bytes": 0.0},
            "rankk": {"ms": 150.0, "launches": 300, "flops": 1e13, "bytes": 1e11},
            "gemv": {"ms": 200.0, "launches": 1000, "flops": 1e12, "bytes": gemv_bytes},
            "resid": {"ms": 10.0, "launches": 40, "flops": 0.0, "bytes": 1e10}}


def test_roofline_even_subdomains():
    n = 1024
    sub_nodes = np.full(n, 729)
    sub_exp = np.full(n, bench.explicit_values_per_sub(772, 730, 42))
    regions = {"linearize": {"launches": 10, "ms": 400.0}}
    main, other = bench.roofline(_prof(1.0e12), regions, {"name": "slab128"}, "mixed", True, sub_nodes, sub_exp)
    parts = dict(other, **{("factorisation" if main["bound"] == "tensor" else "krylov"): main})
    f, k = parts["factorisation"], parts["krylov"]
    pk = bench.peaks()
    # factorisation: algorithmic flops per Jacobian / the class's time
    assert f["algorithmic_flops_per_jacobian"] == pytest.approx(n * bench.factor_flops_per_sub(8))
    assert f["achieved"] == pytest.approx(n * bench.factor_flops_per_sub(8) * 10 / 0.300 / 1e12)
    assert f["frac"] == pytest.approx(f["achieved"] / f["peak"])
    # Krylov: two launches per iteration, packed explicit operators (fewer than the banded factors)
    per_launch = sub_exp.sum() * 4 / 2
    assert k["algorithmic_bytes_per_launch"] == pytest.approx(per_launch)
    assert k["achieved"] == pytest.approx(per_launch * 1000 / 0.200 / 1e9)
    assert k["peak"] == pk.get("hbm_gbs", 6800.0)
    assert "packed lower triangles" in k["work"]


def test_roofline_uneven_caps_at_library_work():
    sub_nodes = np.array([729, 300, 64, 1000] * 50)
    regions = {"linearize": {"launches": 5, "ms": 100.0}}
    tiny = 1.0e6  # launches that read far less than the box model: the model is capped to them
    main, other = bench.roofline(_prof(tiny), regions, {"name": "shell"}, "mixed", True, sub_nodes, None)
    k = main if main["bound"] == "hbm" else other["krylov"]
    assert k["algorithmic_bytes_per_launch"] == pytest.approx(tiny / 1000)
    assert "capped" in k["work"]


def test_traffic_dropped_when_the_source_changes():
    name = "k_symv_batched"
    saved = dict(bench.TRAFFIC[name])
    try:
        assert bench.traffic(name, 1e9) == pytest.approx(saved["dram_per_library_byte"] * 1e9)
        bench.TRAFFIC[name]["sha"] = "0" * 16
        assert bench.traffic(name, 1e9) is None
    finally:
        bench.TRAFFIC[name] = saved
