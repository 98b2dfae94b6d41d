import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # Without a GPU the gpu-marked tests are skipped rather than failing at import.
    try:
        import torch
        have_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        have_gpu = False
    if have_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Filter decisions that differ between the GPU and the oracle: for every parity comparison of
    the run, the entries stored by one side only and the largest of them against the drop
    threshold (the bar allows magnitudes up to 2 t)."""
    try:
        from tests._compare import DROP_FLIPS
    except Exception:  # pragma: no cover
        return
    if not DROP_FLIPS:
        return
    tr = terminalreporter
    tr.write_sep("-", "drop decisions that differ from the oracle (only_gpu / only_oracle / worst |v| / t)")
    total_g = sum(r["only_gpu"] for r in DROP_FLIPS)
    total_o = sum(r["only_oracle"] for r in DROP_FLIPS)
    for r in DROP_FLIPS:
        if r["only_gpu"] or r["only_oracle"]:
            ratio = r["worst_flip"] / r["t_drop"] if r["t_drop"] else 0.0
            tr.write_line(f"n={r['nnz_oracle']:>10} stored: only_gpu={r['only_gpu']} only_oracle={r['only_oracle']} "
                          f"worst/t={ratio:.3f}")
    tr.write_line(f"{len(DROP_FLIPS)} comparisons, {total_g} GPU-only and {total_o} oracle-only entries in total")
