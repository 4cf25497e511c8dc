"""Host logic of the paired inner substeps and of moving meshes (no GPU):
tests/plan_check.cpp prepares a mesh as the library does and checks the
block plans (every node of R in exactly one core; a block's halo is exactly
the P neighbours of its core outside it; each adjacency entry names its P
neighbour's row; k x k cores on a uniform R) and the tables of a mesh whose
vertices move with the draw (directed weight rows, entry ids in the tables,
each entry's undirected edge, every free node's elements, 1/m = 1, the
modes in the internal node order)."""
import os
import shutil
import struct
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    if shutil.which("g++") is None:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("plan") / "plan_check")
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", exe, os.path.join(ROOT, "tests", "plan_check.cpp"),
                    os.path.join(ROOT, "paper_2106_11117_gb300", "csrc", "mesh_prep.cpp")], check=True)
    return exe


def _write(path, m, psi, disp):
    with open(path, "wb") as f:
        f.write(struct.pack("<qqi", m.n_nodes, m.n_tri, psi.shape[1]))
        f.write(np.ascontiguousarray(m.xy, np.float64).tobytes())
        f.write(np.ascontiguousarray(m.tri, np.int32).tobytes())
        f.write(np.ascontiguousarray(m.dirichlet, np.uint8).tobytes())
        f.write(np.ascontiguousarray(m.P, np.uint8).tobytes())
        f.write(np.ascontiguousarray(psi, np.float64).tobytes())
        f.write(np.ascontiguousarray(disp, np.float64).tobytes())


def test_plans_on_a_refined_square(checker, tmp_path):
    from gpu_common import small_level
    lev = small_level(n=16, p=8, K=4, box=(0.3, 0.7, 0.3, 0.7))
    m = lev["mesh"]
    disp = np.zeros((m.n_nodes, 2))
    disp[:, 1] = np.sin(np.pi * m.xy[:, 0]) * 1e-3
    _write(tmp_path / "m.bin", m, lev["psi"], disp)
    out = subprocess.run([checker, str(tmp_path / "m.bin"), "uniform"], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout


def test_plans_on_the_channel(checker, tmp_path):
    from workload.channel import channel_mesh, displacement_mode
    m = channel_mesh(20, 0)
    _write(tmp_path / "c.bin", m, np.zeros((m.n_tri, 1)), displacement_mode(m))
    out = subprocess.run([checker, str(tmp_path / "c.bin")], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "OK", out.stdout
