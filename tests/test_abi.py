"""Host-side checks of the C-ABI library (no GPU needed): it loads, exports every entry
point include/mfmc.h declares, and validates model descriptors on the host."""
import ctypes
import os
import re
import subprocess

import pytest

from tests.conftest import ROOT

HEADER = os.path.join(ROOT, "include", "mfmc.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2310_10750_gb300 import build
    path = build.build()
    from paper_2310_10750_gb300 import mfmc
    return path, mfmc


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(mfmc_\w+)\s*\(", text)
    return sorted(set(n for n in names if not n.endswith("_t")))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mfmc_model_create", "mfmc_model_destroy", "mfmc_solve_batch", "mfmc_solve_fields",
                     "mfmc_plan", "mfmc_estimate", "mfmc_run", "mfmc_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    path, _ = lib
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = set(line.split()[-1] for line in out.splitlines() if line.strip())
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    L = ctypes.CDLL(path)
    for n in declared_functions():
        assert hasattr(L, n)


def test_model_validation_on_host(lib):
    _, mfmc = lib
    m = mfmc.Model(n=64, delta=4 / 64, eps=0.03)
    info = m.info()
    assert info.R == 4 and info.disc_points == 49
    # lattice c_gamma of the constant kernel: 8 eps^2/(pi delta^4) h^2 |D|
    assert info.c_gamma == pytest.approx(8 * 0.03 ** 2 / (3.141592653589793 * (4 / 64) ** 4) / 64 ** 2 * 49)
    assert info.c_gamma == pytest.approx(1.7968, abs=1e-4)
    # beta2 > 0: the active-set solver, chosen by AUTO or named
    b2 = mfmc.Model(n=64, delta=4 / 64, beta2=0.05)
    mfmc.Model(n=64, delta=4 / 64, beta2=0.05, algo=mfmc.ALGO_ACTIVE_SET)
    # no solve yet: the iteration totals are zero and no device memory is read
    assert mfmc.mfmc_model_solver_stats(b2) == (0, 0)
    assert mfmc.mfmc_model_solver_stats(m) == (0, 0)
    assert mfmc._L.mfmc_model_solver_stats(None, None, None) == mfmc.MFMC_EINVAL
    # iteration bounds of the beta2 > 0 solver: host-side validation
    b2.set_iteration_limits(3, 7)
    b2.set_iteration_limits()
    for bad in ((-1, 0), (0, -1), (100001, 0)):
        with pytest.raises(mfmc.MfmcError) as e:
            b2.set_iteration_limits(*bad)
        assert e.value.status == mfmc.MFMC_EINVAL
    assert mfmc._L.mfmc_model_set_iteration_limits(None, 1, 1) == mfmc.MFMC_EINVAL
    # a non-integer delta/h: the disc is { |z| <= 4.5 } and only the generic kernel serves it
    g = mfmc.Model(n=64, delta=4.5 / 64, eps=0.03)
    assert g.info().R == 4
    assert g.info().disc_points == sum(1 for a in range(-4, 5) for b in range(-4, 5) if a * a + b * b <= 20.25)
    for algo in (mfmc.ALGO_PREFIX_TMA, mfmc.ALGO_PREFIX, mfmc.ALGO_RESIDENT, mfmc.ALGO_ROWS, mfmc.ALGO_PREFIX_KAHAN):
        with pytest.raises(mfmc.MfmcError):
            mfmc.Model(n=64, delta=4.5 / 64, algo=algo)
    for bad in (dict(n=62, delta=4 / 62), dict(n=64, delta=33 / 64),
                dict(n=64, delta=4 / 64, tau=0.0), dict(n=64, delta=4 / 64, beta2=-0.05),
                dict(n=64, delta=4 / 64, beta2=0.05, bc=1), dict(n=64, delta=4 / 64, beta2=0.05, algo=1),
                dict(n=64, delta=4 / 64, beta1=0.0), dict(n=64, delta=4 / 64, nsteps=-1),
                dict(n=64, delta=4 / 64, kernel=1, delta_hf=0.0), dict(n=8, delta=4 / 8),
                dict(n=64, delta=4 / 64, ic_base_n=96), dict(n=64, delta=4 / 64, algo=9)):
        with pytest.raises(mfmc.MfmcError) as e:
            mfmc.Model(**bad)
        assert e.value.status == mfmc.MFMC_EINVAL
        assert mfmc.mfmc_last_error()
    # the resident form needs the field in shared memory: n = 1024 is rejected
    with pytest.raises(mfmc.MfmcError):
        mfmc.Model(n=1024, delta=32 / 1024, algo=mfmc.ALGO_RESIDENT)


def test_host_eps_resolution_matches_oracle_generator(lib):
    _, mfmc = lib
    import numpy as np
    import oracle
    m = mfmc.Model(n=64, delta=4 / 64, eps=0.03, eps_lo=0.024, eps_hi=0.036)
    seeds = np.arange(20) + 20231016
    got = mfmc.mfmc_sample_eps(m, seeds)
    ref = oracle.OracleModel(n=64, delta=4 / 64, eps_lo=0.024, eps_hi=0.036)
    assert [ref.sample_eps(int(s)) for s in seeds] == got.tolist()


def test_host_setters_and_version(lib):
    _, mfmc = lib
    assert mfmc.mfmc_version()
    m = mfmc.Model(n=256, delta=8 / 256, eps=0.02)
    for v in range(11):
        m.set_tile_variant(v)
        assert m.info().tile_variant == v
    for v in (-1, 11):
        with pytest.raises(mfmc.MfmcError) as e:
            m.set_tile_variant(v)
        assert e.value.status == mfmc.MFMC_EINVAL
    assert m.info().tile_variant == 10           # a rejected call changes nothing
    m.set_band_height(64, 4)
    assert (m.info().band_height, m.info().columns_per_thread) == (64, 4)
    for rows, cols in ((7, 4), (16385, 4), (64, 2), (64, 3), (-1, 4)):
        with pytest.raises(mfmc.MfmcError) as e:
            m.set_band_height(rows, cols)
        assert e.value.status == mfmc.MFMC_EINVAL
    assert (m.info().band_height, m.info().columns_per_thread) == (64, 4)
    m.set_band_height(0, 4)                      # 0: the batch's rows split evenly over the warps
    assert m.info().band_height == 0


def test_trace_argument_checks_on_host(lib):
    # rejected before any device call, so these run without a GPU
    _, mfmc = lib
    assert mfmc._L.mfmc_trace_enable((1 << 28) + 1) == mfmc.MFMC_EINVAL
    assert "2^28" in mfmc.mfmc_last_error()
    assert mfmc._L.mfmc_trace_read(None, 5, None, None) == mfmc.MFMC_EINVAL


STRUCTS = ["mfmc_model_desc", "mfmc_sample_params", "mfmc_model_info", "mfmc_plan_t", "mfmc_server_stats",
           "mfmc_trace_record"]


def test_binding_struct_layouts_match_the_header(lib, tmp_path):
    # The ctypes mirrors of the boundary's structs must have the C compiler's size and field
    # offsets for include/mfmc.h (a field added, dropped or reordered on one side only would
    # shift every field after it).  Compiled as C by gcc on the host, no GPU.
    _, mf = lib
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "mfmc.h"', 'int main(void) {']
    for s in STRUCTS:
        lines.append(f'    printf("{s} %zu\\n", sizeof({s}));')
        for name, _ in getattr(mf, s)._fields_:
            lines.append(f'    printf("{s}.{name} %zu\\n", offsetof({s}, {name}));')
    lines += ['    return 0;', '}']
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                       text=True).stdout.splitlines())
    for s in STRUCTS:
        cls = getattr(mf, s)
        assert int(got[s]) == ctypes.sizeof(cls), s
        for name, _ in cls._fields_:
            assert int(got[f"{s}.{name}"]) == getattr(cls, name).offset, (s, name)


def test_binding_signatures_match_the_header(lib):
    # every entry point the header declares has a binding whose argument count and return
    # kind (status, void, string) are the declaration's
    _, mf = lib
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    decls = re.findall(r"(mfmc_status|void|const char\s*\*)\s*(mfmc_\w+)\s*\(([^;{]*?)\)\s*;", text)
    assert sorted(d[1] for d in decls) == declared_functions()
    for ret, name, params in decls:
        p = params.strip()
        nargs = 0 if p in ("", "void") else p.count(",") + 1
        f = getattr(mf._L, name)
        assert f.argtypes is not None and len(f.argtypes) == nargs, name
        want = {"mfmc_status": ctypes.c_int, "void": None}.get(ret, ctypes.c_char_p)
        assert f.restype is want, (name, f.restype)
