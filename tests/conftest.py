import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

GOLDEN = os.path.join(ROOT, "tests", "golden")


class OoiErrors:
    """Per-sample errors of the GPU path against the FP64 oracle, gathered by the parity tests
    per workload and printed at the end of the run: the OoI f = (1 + mean u) / 2 relative, the
    mean of u absolute and the field max-norm (where the test compares fields)."""

    def __init__(self):
        self.rows = {}

    def add(self, workload, f_gpu, f_orc, mean_gpu=None, mean_orc=None, field_err=None):
        r = self.rows.setdefault(workload, [0, 0.0, None, None])
        r[0] += 1
        r[1] = max(r[1], abs(float(f_gpu) - float(f_orc)) / abs(float(f_orc)))
        if mean_gpu is not None:
            e = abs(float(mean_gpu) - float(mean_orc))
            r[2] = e if r[2] is None else max(r[2], e)
        if field_err is not None:
            r[3] = float(field_err) if r[3] is None else max(r[3], float(field_err))


_OOI_ERRORS = OoiErrors()


@pytest.fixture(scope="session")
def ooi_errors():
    return _OOI_ERRORS


def pytest_terminal_summary(terminalreporter):
    rows = _OOI_ERRORS.rows
    if not rows:
        return
    tr = terminalreporter
    tr.write_line("per-sample error against the FP64 oracle (max over the samples checked; target 1e-5 rel. on f):")
    for w, (k, rel, mean, field) in rows.items():
        extra = "" if mean is None else f", mean u {mean:.1e} abs"
        extra += "" if field is None else f", field {field:.1e} abs"
        tr.write_line(f"  {w}: {k} samples, f {rel:.1e} rel{extra}")


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")


def read_golden(name):
    """Rows of a whitespace-separated golden file, comments dropped."""
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.fixture(scope="session")
def gpu_lib():
    """The CUDA library, built in-tree if needed.  GPU tests only."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test collected on a machine without CUDA")
    from paper_2310_10750_gb300 import build as pkg_build
    pkg_build.build()
    from paper_2310_10750_gb300 import mfmc
    return mfmc
