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
    assert cfg == {"chain_reduction": False, "locality_order": False, "early_termination_orders": 0,
                   "pipeline": "automatic"}


def test_spmm_traffic_reads_the_line_of_its_width(tmp_path):
    """The roofline's traffic comes from the committed summary line of the
    bench's block width, only while the SpMM source has the recorded hash."""
    import hashlib
    b = _bench()
    kern = tmp_path / "k.cu"
    kern.write_text("kernel source")
    sha = hashlib.sha256(b"kernel source").hexdigest()
    summ = tmp_path / "s.md"
    summ.write_text("x\ntraffic_bytes_per_launch: 8.5e9 source_sha256: %s width: 64\n"
                    "traffic_bytes_per_launch: 3.1e9 source_sha256: %s width: 32\n"
                    "traffic_bytes_per_launch: 1.0e9 source_sha256: %s width: 16\n" % (sha, sha, "0" * 64))
    assert b.spmm_traffic(64, str(kern), str(summ)) == (8.5e9, str(summ))
    assert b.spmm_traffic(32, str(kern), str(summ)) == (3.1e9, str(summ))
    v, why = b.spmm_traffic(16, str(kern), str(summ))
    assert v is None and "changed" in why
    v, why = b.spmm_traffic(8, str(kern), str(summ))
    assert v is None and "width 8" in why
