"""The C ABI used from plain C (tests/c/sbim_c_client.c, no PyTorch): the
client is compiled with nvcc against include/sbim.h and the in-tree
libsbim.so, steps a half-space through a seeded history with device buffers
(sbim_step) and host buffers (sbim_step_host), and its tractions match the
FP64 oracle within the FP32 bound; the two entry points agree to within the
rounding of the lag-0 addition, which the host-buffer step makes last."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from oracle.sbim_oracle import SBIMOracle
from paper_2102_08756_gb300.synth import separable_history
from tests._errors import Worst, assert_finite

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CS, CP, RHO = 3464.0, 6000.0, 2670.0


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    libdir = os.path.join(ROOT, "paper_2102_08756_gb300", "_lib")
    exe = str(tmp_path_factory.mktemp("c") / "sbim_c_client")
    subprocess.run([nvcc, "-O2", "-o", exe, os.path.join(ROOT, "tests", "c", "sbim_c_client.c"),
                    "-I", os.path.join(ROOT, "include"), "-L", libdir, "-lsbim",
                    "-Xlinker", "-rpath=" + libdir], check=True, capture_output=True)
    return exe


@pytest.mark.parametrize("n1,n3,n_cut,side,steps", [(24, 16, 9, 1, 20), (32, 32, 40, -1, 30)])
def test_c_client_matches_oracle(client, tmp_path, n1, n3, n_cut, side, steps):
    dx = 100.0
    dt = 0.3 * dx / CP
    L1, L3 = n1 * dx, n3 * dx
    hist = separable_history(n1, n3, L1, L3, steps, dt, CS, seed=n1 + steps, spectrum="k2")
    src, dst = tmp_path / "in.bin", tmp_path / "out.bin"
    with open(src, "wb") as f:
        np.array([n1, n3, n_cut, side, steps], dtype=np.int32).tofile(f)
        np.array([L1, L3, CS, CP, RHO, dt], dtype=np.float64).tofile(f)
        for m in range(steps):
            hist.u(m).astype(np.float32).tofile(f)
            hist.v(m).astype(np.float32).tofile(f)
    r = subprocess.run([client, str(src), str(dst)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    out = np.fromfile(dst, dtype=np.float32).reshape(steps, 2, 3, n3, n1)
    o = SBIMOracle(n1, n3, L1, L3, CS, CP, RHO, dt, n_cut, side)
    assert_finite(out, "client output")
    worst = Worst()
    for m in range(steps):
        # host buffers: the lag-0 term is added after the other lags
        assert np.abs(out[m, 0] - out[m, 1]).max() <= 1e-6 * np.abs(out[m, 0]).max()
        ref = o.step(hist.u(m).astype(np.float32).astype(np.float64),
                     hist.v(m).astype(np.float32).astype(np.float64))["tau"]
        for c in range(3):
            nr = np.linalg.norm(ref[c])
            if nr > 0:
                worst.update(np.linalg.norm(out[m, 0, c] - ref[c]) / nr)
    assert worst.value < 1e-5, worst
