"""CPU-only checks of the C ABI: the library builds and loads, exports every
entry point that include/pdds.h declares, and its host-side geometry (no
CUDA call) agrees with the oracle's knots and CSR pattern (Sec. 3.1)."""
import os
import re

import numpy as np
import pytest

from paper_2301_05780_gb300 import pdds, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pdds_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    L = pdds.lib()
    decl = declared_functions()
    assert len(decl) >= 15
    for name in decl:
        assert hasattr(L, name), name
    assert set(decl) == set(pdds.exported_names())


@pytest.mark.parametrize("grid", [
    W.config1().grid,
    W.config2().grid,
    dict(x0=-1.0, x1=2.0, y0=0.5, y1=2.5, Hx=3, Hy=2, m=4, ext=1),
    dict(x0=0.0, x1=4.0, y0=0.0, y1=4.0, Hx=5, Hy=5, m=8, ext=4),
    dict(x0=0.0, x1=1.0, y0=0.0, y1=1.0, Hx=1, Hy=3, m=5, ext=2),
    dict(x0=0.0, x1=1.0, y0=0.0, y1=1.0, Hx=4, Hy=4, m=1, ext=0),
])
def test_host_geometry_matches_oracle(orc, grid):
    xy, rp, col = pdds.pdds_geometry_host(grid)
    P = orc.Problem(grid, 4, params=(1.4, 0, 0, 0, 0, 0))
    assert xy.shape[0] == P.n
    assert np.allclose(xy, P.xy, rtol=0, atol=1e-12)
    assert np.array_equal(rp, P.row_ptr)
    assert np.array_equal(col, P.col)


def test_config_knot_counts():
    """Knot counts of the five workloads (config 4: 124,929 unique knots)."""
    for w, n in [(W.config1(), 29), (W.config2(), 833), (W.config4(with_tables=False), 124929),
                 (W.config5(), 113665)]:
        xy, rp, col = pdds.pdds_geometry_host(w.grid)
        assert xy.shape[0] == n, w.name


@pytest.mark.parametrize("bad", [
    dict(x0=0, x1=0, y0=0, y1=1, Hx=2, Hy=2, m=4, ext=1),
    dict(x0=0, x1=1, y0=0, y1=1, Hx=1, Hy=1, m=4, ext=1),
    dict(x0=0, x1=1, y0=0, y1=1, Hx=2, Hy=2, m=0, ext=1),
    dict(x0=0, x1=1, y0=0, y1=1, Hx=2, Hy=2, m=4, ext=-1),
])
def test_host_geometry_rejects_invalid_grids(bad):
    with pytest.raises(pdds.PddsError) as e:
        pdds.pdds_geometry_host(bad)
    assert e.value.status == pdds.PDDS_EINVAL
    assert "grid" in str(e.value)


def test_record_and_struct_layouts_match_the_header(tmp_path):
    """The binding's record dtype and structs have the sizes the C header gives
    (compiled with the host C compiler, no CUDA)."""
    src = tmp_path / "sz.c"
    src.write_text('#include <stdio.h>\n#include "pdds.h"\nint main(void){printf("%zu %zu %zu %zu",'
                   ' sizeof(pdds_path_record), sizeof(pdds_grid), sizeof(pdds_coeffs),'
                   ' sizeof(pdds_stats_t)); return 0;}\n')
    exe = tmp_path / "sz"
    import subprocess
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    rec, grid, coeffs, stats = map(int, subprocess.run([str(exe)], capture_output=True, text=True,
                                                       check=True).stdout.split())
    import ctypes
    assert rec == pdds.RECORD_BYTES == 40
    assert grid == ctypes.sizeof(pdds.pdds_grid)
    assert coeffs == ctypes.sizeof(pdds.pdds_coeffs)
    assert stats == ctypes.sizeof(pdds.pdds_stats_t)


def test_null_arguments_are_rejected_before_any_cuda_call():
    """Argument checks that precede every CUDA call (so they run on a machine
    without a GPU): a NULL context or NULL device pointers give EINVAL."""
    L = pdds.lib()
    assert L.pdds_set_network_engine(None, pdds.NET_TCGEN05) == pdds.PDDS_EINVAL
    assert L.pdds_set_philox_tag(None, 0) == pdds.PDDS_EINVAL
    assert L.pdds_set_wait_limit(None, 1.0) == pdds.PDDS_EINVAL
    assert L.pdds_mlp_loss_grad(None, None, None, 10, None, None, None) == pdds.PDDS_EINVAL
    assert L.pdds_mlp_loss_grad_tc(None, None, None, 10, None, None, None) == pdds.PDDS_EINVAL
    assert L.pdds_mlp_train_tc(None, None, None, 10, 5, 1e-3, None, None) == pdds.PDDS_EINVAL
    assert L.pdds_mlp_train(None, None, None, 10, 5, 1e-3, None, None) == pdds.PDDS_EINVAL
