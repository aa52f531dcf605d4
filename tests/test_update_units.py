"""Host check of the tensor-core trailing update's unit enumeration.

The update kernel walks one flat list of units per launch: single 128 x 128
tiles for the next outer block's columns, pairs of tiles of one tile row
(128 x 256, sharing the W operand) elsewhere.  tests/units_check.cu compiles
the enumeration the kernel uses (tc_update.cuh) into a host program that
checks every window shape covers each tile of its lower part exactly once,
and that the backward substitution's split of an ancestor-row product into
parts covers every row with at most BWD_PARTS_MAX non-empty parts.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_units_cover_every_tile_once(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "units_check")
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-o", exe,
                    os.path.join(HERE, "units_check.cu")], check=True, capture_output=True, timeout=300)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.startswith("ok"), out.stdout + out.stderr
