"""The tile orders of the tensor-core GEMM launches (csrc/tile_order.cuh),
compiled for the host with g++ and checked by tests/tile_order_check.cpp:
every launch form (single CTAs over all or a range of tiles, CTA pairs
sharing the P panel) visits each tile it owns exactly once, inside
the grid, and the split launches of the host-buffer call cover the same
tiles as the whole launch.  No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tile_orders_cover_every_tile_once(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    exe = str(tmp_path / "tile_order_check")
    subprocess.run([gxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_2403_06937_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "tile_order_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout
    assert "tile orders ok" in out.stdout
