"""Host logic of bench.py: both arms describe the same workload and PCG stop rule in
`config` (the reference arm adds only the oracle's own FP64 rule)."""
import argparse

import bench


def _w():
    return {"n": 100_000, "d": 10_000, "s": 200, "rho": 70.0, "rho_extra": 100.0, "pcg_tol": 1e-4,
            "pcg_beta": 1.75, "pcg_tol_fp64": 1e-8}


def test_default_rule_is_the_decaying_schedule():
    ap_args = argparse.Namespace(pcg_tol=None, pcg_mode="rnorm_pow")
    w = _w()
    bench.apply_pcg_args(w, ap_args)
    assert w["pcg_tol"] == 1.75 and w["pcg_mode"] == "rnorm_pow"
    assert "k^beta with beta = 1.75" in bench.workload_config(w)["pcg"]


def test_explicit_tolerance_and_rel_mode():
    w = _w()
    bench.apply_pcg_args(w, argparse.Namespace(pcg_tol=3e-4, pcg_mode="rel"))
    assert w["pcg_tol"] == 3e-4
    assert bench.workload_config(w)["pcg"].startswith("f32, rel-tol 0.0003")
    w = _w()
    bench.apply_pcg_args(w, argparse.Namespace(pcg_tol=2.5, pcg_mode="rnorm_pow"))
    assert "beta = 2.5" in bench.workload_config(w)["pcg"]


def test_both_arms_share_the_workload_config():
    a, b = _w(), _w()
    for w in (a, b):
        bench.apply_pcg_args(w, argparse.Namespace(pcg_tol=None, pcg_mode="rnorm_pow"))
    assert bench.workload_config(a) == bench.workload_config(b)
    assert bench.workload_config(a)["rho"] == 70.0
