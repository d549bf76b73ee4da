import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU and the compiled libwsm")
    config.addinivalue_line("markers", "slow: longer CPU-only checks")


def golden(name: str) -> str:
    return os.path.join(ROOT, "tests", "golden", name)


def read_golden(name: str) -> list[list[str]]:
    rows = []
    with open(golden(name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def pytest_terminal_summary(terminalreporter):
    """List the whole runs the GPU parity tests compared with the oracle and
    the pass at which each first met a decision taken by FP32 rounding."""
    mod = sys.modules.get("parity")
    if mod is None or not mod.RUNS:
        return
    terminalreporter.section("whole-path parity runs (GPU vs oracle)")
    for name, it_g, it_o, div, rel in mod.RUNS:
        where = "no divergence" if div is None else f"first rounding decision at pass {div}"
        terminalreporter.write_line(f"{name}: iterations {it_g}/{it_o}, {where}, "
                                    f"free-run MSE relative difference {rel:.2e}")
