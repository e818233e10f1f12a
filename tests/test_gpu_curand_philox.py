"""The oracle's Philox4x32-10 against cuRAND's device implementation (an
independent library generator run on the GPU), over random counters and keys,
including counters whose high words are set (the trajectory and step bits above
32 of the keyed contract)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_oracle_philox_equals_curand(oracle_mod, tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "curand_philox"
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2",
                    os.path.join(HERE, "cuda", "curand_philox.cu"), "-o", str(exe)], check=True)
    rng = np.random.default_rng(2024)
    rows = rng.integers(0, 2**32, size=(200, 6), dtype=np.uint64)
    rows[:, 3] %= 2**30       # cuRAND takes the block counter's low 64 bits as an output
                              # offset (4 outputs per block), so c1 < 2^30 is expressible
    rows[:50, 5] = 0          # zero high counter words (small subsequences)
    rows[50:60, :2] = 0       # zero keys
    text = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
    out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout
    got = np.array([[int(v) for v in line.split()] for line in out.splitlines()], dtype=np.uint64)
    assert got.shape == (200, 4)
    for r, g in zip(rows, got):
        key = [int(r[0]), int(r[1])]
        ctr = [int(r[2]), int(r[3]), int(r[4]), int(r[5])]
        assert [int(x) for x in oracle_mod.philox(ctr, key)] == [int(x) for x in g], (ctr, key)
