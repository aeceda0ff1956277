"""The persistent scheduler's task graph (Section 3.2, Fig. 2: window tasks
and left / right update tasks in a sequentially consistent order), checked
on the host: tests/graph_check.cpp is compiled with the library's planner
source and run on seeded block structures and sweep plans.  Every
dependence goes forward, every pair of overlapping tasks (same matrix) is
ordered, every tile follows its window task, and the queue order is
topological; for reorderings, the cuts of the chunked launches keep every
pair of overlapping windows in planner order and each chunk's graph passes
the same checks."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_04975_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("graph") / "graph_check")
    subprocess.run([nvcc, "-O2", "-std=c++17", "-x", "cu", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "graph_check.cpp"), os.path.join(CSRC, "plan.cu"),
                    "-o", out], check=True)
    return out


def run(checker, *args):
    p = subprocess.run([checker] + [str(a) for a in args], capture_output=True, text=True,
                       timeout=120)
    assert p.returncode == 0 and p.stdout.startswith("OK"), p.stdout + p.stderr
    return p.stdout


@pytest.mark.parametrize("n,w,m,q,z", [(40, 8, 3, 1, 0), (120, 16, 6, 1, 0), (300, 64, 30, 1, 0),
                                       (300, 32, 12, 0, 0), (200, 24, 10, 1, 1), (257, 64, 32, 1, 1),
                                       (600, 256, 128, 1, 0), (500, 200, 40, 1, 0)])
@pytest.mark.parametrize("seed", [1, 2])
def test_reordering_graph(checker, n, w, m, q, z, seed):
    run(checker, n, w, m, q, z, seed, 0)


@pytest.mark.parametrize("n,w,nb", [(50, 16, 2), (200, 48, 8), (300, 64, 16), (97, 24, 3)])
def test_sweep_graph(checker, n, w, nb):
    run(checker, n, w, nb, 1, 0, 0, 1)
