"""bench.py's modes exist and its options parse (no device work): every
workload named on the command line dispatches to a defined function."""
import importlib.util
import os

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_every_mode_has_its_function():
    b = _bench()
    for name in ["run_blackbox_only", "run_batch", "run_serve", "run_sigma_only", "run_reference", "main",
                 "apply_options", "options_config", "cpu_baseline"]:
        assert callable(getattr(b, name, None)), name
    src = open(os.path.join(ROOT, "bench.py")).read()
    for flag in ["--workload", "--chain-reduction", "--locality-order", "--early-termination", "--only-blackbox",
                 "--only-sigma", "--impl"]:
        assert flag in src, flag


def test_options_config_defaults_off():
    import argparse
    b = _bench()
    cfg = b.options_config(argparse.Namespace())
    assert cfg == {"chain_reduction": False, "locality_order": False, "early_termination_orders": 0}
