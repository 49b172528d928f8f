"""Bounds-checked build: every index the step kernels compute (list entries, neighbour nodes,
storage slots, inlet/outlet rows, adhesion targets) is checked against its buffer, and an index
outside it sets a device error flag instead of touching memory.  The library is rebuilt with
-DLBM_BOUNDS_CHECK into its own directory and a representative set of parity cases (walls and
periodic axes, inlet/outlet, MRT with dissolution flips and list rebuilds, deposition,
two components with adhesion, reduced storage, the velocity inlet and the temperature-dependent
reaction (the full kernel variant), ensembles) runs against it in a child process;
each comparison first synchronises, so any out-of-range index fails the case."""
import os
import subprocess
import sys

import pytest

from paper_2502_12955_gb300 import build as lbm_build

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [
    "test_gpu_parity.py::test_2d_all_scalar_features",
    "test_gpu_parity.py::test_3d_bgk_walls_and_scalars",
    "test_gpu_parity.py::test_3d_mrt_dissolution_with_flips",
    "test_gpu_parity.py::test_2d_deposition_with_flips",
    "test_gpu_parity.py::test_3d_deposition_inlet",
    "test_gpu_parity.py::test_two_component_3d_with_solid_and_adhesion",
    "test_gpu_parity.py::test_pops_roundtrip_and_odd_layout",
    "test_gpu_parity.py::test_reduced_precision_against_fp64_oracle",
    "test_gpu_parity.py::test_velocity_inlet_channel",
    "test_gpu_parity.py::test_temperature_dependent_reaction_with_heat",
    "test_gpu_ensemble.py",
]


def test_parity_cases_under_bounds_checked_build():
    out = os.path.join(lbm_build.BUILD, "bounds_checked")
    lib = lbm_build.build(out_dir=out, extra_flags=["-DLBM_BOUNDS_CHECK"])
    env = dict(os.environ, LBM_LIBRARY=lib)
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider"]
    cmd += [os.path.join(ROOT, "tests", c) for c in CASES]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert "LBM_ERR_BOUNDS" not in tail
