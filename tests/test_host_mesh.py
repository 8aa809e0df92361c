"""The library's host-side mesh (C++) against the oracle (CPU only): same
macro mesh, canonical node order, positions and Dirichlet flags."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle import mesh as M

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def dumper(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    out = str(tmp_path_factory.mktemp("bin") / "mesh_dump")
    src = [os.path.join(ROOT, "tests/cpp/mesh_dump.cpp"), os.path.join(ROOT, "paper_1608_06473_gb300/csrc/mesh.cpp")]
    cuda_inc = "/usr/local/cuda/include"
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", cuda_inc, *src, "-o", out], check=True)
    return out


@pytest.mark.parametrize("tang,layers,N", [(0, 1, 8), (1, 2, 4), (0, 1, 16)])
def test_positions_order_and_dirichlet(dumper, tmp_path, tang, layers, N):
    path = str(tmp_path / "d.bin")
    subprocess.run([dumper, "0.55", "1.0", str(tang), str(layers), str(N), path], check=True)
    raw = open(path, "rb").read()
    hdr = np.frombuffer(raw[:48], dtype=np.int64)
    nt = int(hdr[0])
    xyz = np.frombuffer(raw[48:48 + 24 * nt], dtype=np.float64).reshape(nt, 3)
    dirich = np.frombuffer(raw[48 + 24 * nt:48 + 25 * nt], dtype=np.uint8).astype(bool)
    cmap = np.frombuffer(raw[48 + 25 * nt:], dtype=np.int64)
    sh = M.make_shell(tang=tang, layers=layers)
    lv = M.make_level(sh, N)
    assert nt == lv.n_total and tuple(hdr[1:5]) == (sh.nV, sh.nE, sh.nF, sh.nC)
    assert np.array_equal(dirich, lv.dirichlet)
    assert np.max(np.abs(xyz - lv.coords)) <= 1e-15
    assert np.array_equal(cmap.reshape(sh.nC, -1), lv.cell_map)
