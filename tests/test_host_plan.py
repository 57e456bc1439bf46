"""The C++ planner's host logic against the oracle (CPU only).

The probe in tests/host/plan_probe.cpp links only the planner (plan.cpp) and
prints its integer description of a discretisation; the oracle's
Discretization fixes the same quantities from Sects. 3-4: the node positions,
the node sets N^(i) of Sect. 4.1 (the planner stores them as contiguous
unrolled ranges, physical node = u mod N_quad), the exactness sets J^(i),
the test functions non-zero at each node, and the collocation nodes of the
collocation form (oracle.collocation.collocation_nodes).
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle.collocation as oc
from oracle.discretization import Discretization

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "host", "plan_probe.cpp")
PLAN = os.path.join(ROOT, "paper_1703_10016_gb300", "csrc", "plan.cpp")
OUT_DIR = os.path.join(HERE, "host", "_build")


@pytest.fixture(scope="module")
def probe():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    os.makedirs(OUT_DIR, exist_ok=True)
    exe = os.path.join(OUT_DIR, "plan_probe")
    r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "include"), "-x", "cu", SRC, PLAN,
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def run(exe, n, d, nref, closed):
    r = subprocess.run([exe, str(n), str(d), str(nref), str(int(closed))], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    out = {}
    for line in r.stdout.splitlines():
        key, *vals = line.split()
        out[key] = np.array([int(v) for v in vals])
    return out


# n from the smallest closed size the library accepts, 2(d + 1), to several tiles
CASES = [(n, d, nref, closed) for closed in (True, False) for d in (2, 3, 4, 5) for nref in (1, 2, 3, 4)
         for n in (2 * (d + 1), 2 * d + 5, 40)]


@pytest.mark.parametrize("n,d,nref,closed", CASES)
def test_planner_matches_oracle(probe, n, d, nref, closed):
    got = run(probe, n, d, nref, closed)
    disc = Discretization(0.0, 1.0, n, d, nref, closed)
    den = int(got["den"][0])
    assert den == 2 * (d + 1)
    np.testing.assert_array_equal(got["pos"], np.rint(disc.node_pos * den).astype(int))
    for i in range(disc.n):
        nodes = set(int(u) % disc.Nq for u in range(got["lo"][i], got["hi"][i] + 1))
        assert nodes == set(int(m) for m in disc.support_nodes(i)), i
    # J^(i): one or two ranges of exactness functions
    for i in range(disc.n):
        js = set(range(got["jlo1"][i], got["jhi1"][i] + 1)) | set(range(got["jlo2"][i], got["jhi2"][i] + 1))
        assert js == set(int(j) for j in disc.overlapping_fine(i)), i
    # node bands: B_{jfirst + r}(eta_m) != 0 exactly for the member bits r (unrolled test index);
    # at a knot the end of a support evaluates to rounding-level values in floating point
    Bt = disc.test_basis(disc.eta)[0]                    # (n, N_quad), cyclic for closed curves
    for m in range(disc.Nq):
        nz = set(int(i) for i in np.nonzero(np.abs(Bt[:, m]) > 1e-12)[0])
        band = set((got["jfirst"][m] + r) % disc.n for r in range(d + 1) if (got["member"][m] >> r) & 1)
        assert band == nz, m
    if closed:
        np.testing.assert_array_equal(got["colloc"], oc.collocation_nodes(disc))
