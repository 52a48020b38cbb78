"""CPU check of the library's RBF cardinal-function tables (no GPU): the
host table builder of libpdds (pdds_rbf.cpp) is compiled with a small driver
(tests/rbf_table_probe.cpp) that evaluates the tables exactly as the path
kernel does; the values must match the oracle's FP64 cardinal functions
(Sec. 2.1, Eq. 5) to the tables' stated bound plus FP32 evaluation, and the
shape parameter for cond(Phi) = 1e10 must match the oracle's."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2301_05780_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cxx = shutil.which("g++")
    cuda_inc = "/usr/local/cuda/include"
    if cxx is None or not os.path.isdir(cuda_inc):
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("rbf") / "probe")
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", cuda_inc, "-I", CSRC, "-I",
                    os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "rbf_table_probe.cpp"),
                    os.path.join(CSRC, "pdds_rbf.cpp"), "-o", exe], check=True)
    return exe


def _run(exe, c, queries):
    inp = f"{float(c)!r}\n" + "".join(f"{L} {float(s)!r}\n" for L, s in queries)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    lines = out.strip().splitlines()
    deg, err = lines[0].split()[1], float(lines[0].split()[3])
    vals = [np.array([float(v) for v in ln.split()]) for ln in lines[1:1 + len(queries)]]
    shape = float(lines[-1].split()[1])
    return int(deg), err, vals, shape


@pytest.mark.parametrize("L,cond", [(23, 1e8), (23, 1e10), (41, 1e10), (145, 1e10)])
def test_tables_match_oracle_cardinals(orc, probe, L, cond):
    c = orc.rbf_shape_for_cond(L, cond)
    rng = np.random.default_rng(L)
    pts = list(rng.uniform(0, L - 1, size=12)) + [0.0, L - 1.0, 0.5, L / 2.0]
    deg, err, vals, shape = _run(probe, c, [(L, s) for s in pts])
    assert err < 1e-5
    for s, H in zip(pts, vals):
        ref = orc.rbf_cardinal(L, c, s)
        assert np.abs(H - ref).max() < 2e-5, (s, np.abs(H - ref).max())
    assert shape == pytest.approx(orc.rbf_shape_for_cond(L, 1e10), rel=1e-6)
