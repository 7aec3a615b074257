"""The factorization's and the traversal's host planning without a GPU.

The library's host sources (factor.cu, solve.cu and emu_plan.cpp, compiled
as C++, with analyze.cpp) are linked against test doubles of the CUDA runtime
and of every kernel launch (tests/host_planning/device_doubles.cpp).  Each
launch double reads the task arrays the host uploaded and checks them against
what its kernel reads: every output tile inside its block, every term range
inside the launch's terms, operands stored with leading dimensions that hold
them, copy tasks consistent with their mode, and for the emulated products
every digit block, exponent and flag the product kernel addresses inside the
split of its own operand and inside the launch's workspace, in at most 512 K
chunks.  Ranks read back from the "device" are a constant, so the symbolic
program of Algorithm 1 runs with blocks of realistic sizes.  The same
scenario planned twice gives the same task arrays (the digest of all of them),
so the launches do not depend on hashing or allocation order.
"""
import os
import re
import shutil
import subprocess
import concurrent.futures as cf

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1510_07363_gb300", "csrc")
HERE = os.path.join(ROOT, "tests", "host_planning")
LIB_SOURCES = ["factor.cu", "solve.cu", "emu_plan.cpp", "analyze.cpp"]
TEST_SOURCES = ["device_doubles.cpp", "scenario.cpp"]


def cuda_include():
    for nvcc in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if nvcc and os.path.exists(nvcc):
            inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(nvcc))), "include")
            if os.path.exists(os.path.join(inc, "cuda_runtime.h")):
                return inc
    return None


@pytest.fixture(scope="module")
def scenario_exe(tmp_path_factory):
    cxx = shutil.which("g++")
    inc = cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    out = tmp_path_factory.mktemp("host_planning")
    flags = ["-std=c++17", "-O1", "-I" + inc, "-I" + CSRC, "-I" + os.path.join(ROOT, "include"), "-I" + HERE]

    def compile_one(path):
        obj = os.path.join(str(out), os.path.basename(path) + ".o")
        lang = ["-x", "c++"] if path.endswith(".cu") else []
        p = subprocess.run([cxx, *flags, *lang, "-c", path, "-o", obj], capture_output=True, text=True)
        assert p.returncode == 0, p.stderr
        return obj

    paths = [os.path.join(CSRC, s) for s in LIB_SOURCES] + [os.path.join(HERE, s) for s in TEST_SOURCES]
    with cf.ThreadPoolExecutor(max_workers=len(paths)) as ex:
        objs = list(ex.map(compile_one, paths))
    exe = os.path.join(str(out), "scenario")
    p = subprocess.run([cxx, "-o", exe, *objs, "-lpthread"], capture_output=True, text=True)
    assert p.returncode == 0, p.stderr
    return exe


def run(exe, *args):
    p = subprocess.run([exe, *map(str, args)], capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stdout + p.stderr
    return {k: v for k, v in re.findall(r"(\w+)=([0-9a-f]+)", p.stdout)}


# grid (5: 2D, 7: 3D), nx, ny, nz, leaf, rank, symmetric, precision form, emulated products,
# [instances, [separation, [eq. curOff6]]]
SCENARIOS = {
    "poisson3d_16_symmetric": (7, 16, 16, 16, 64, 12, 1, 0, 1),
    "poisson3d_16_general_rank40": (7, 16, 16, 16, 64, 40, 0, 0, 1),
    "poisson2d_12x10_leaf8": (5, 12, 10, 1, 8, 3, 0, 0, 1),
    "poisson3d_32_rank30": (7, 32, 32, 32, 64, 30, 1, 0, 1),
    "poisson3d_16_precision_form": (7, 16, 16, 16, 64, 12, 1, 1, 1),
    "poisson3d_16_fp64_fma": (7, 16, 16, 16, 64, 12, 1, 0, 0),
    "batch_of_4_2d": (5, 40, 48, 1, 64, 8, 0, 0, 1, 4),
    "poisson3d_16_distance3": (7, 16, 16, 16, 64, 12, 1, 0, 1, 1, 3),
    "poisson3d_16_curoff6": (7, 16, 16, 16, 64, 12, 1, 0, 1, 1, 0, 1),
    "poisson3d_24_rank100": (7, 24, 24, 24, 64, 100, 0, 0, 1),
}


@pytest.mark.parametrize("name", list(SCENARIOS))
def test_launch_plans_are_consistent(scenario_exe, name):
    """Every launch of the scenario passes the doubles' checks, and the
    engines are the ones the options select."""
    args = SCENARIOS[name]
    r = run(scenario_exe, *args)
    assert int(r["failures"]) == 0
    assert int(r["eliminations"]) > 0 and int(r["gemm_launches"]) > 0 and int(r["copy_tasks"]) > 0
    fp32, emu = args[7], args[8]
    if fp32:
        assert int(r["tc_launches"]) > 0 and int(r["emu_launches"]) == 0
    elif not emu:
        assert int(r["emu_launches"]) == 0 and int(r["tc_launches"]) == 0
    if emu and not fp32 and name != "poisson2d_12x10_leaf8":   # products of at least 64^3 multiply-adds
        assert int(r["emu_launches"]) > 0 and int(r["emu_splits"]) > 0


def test_planning_is_deterministic(scenario_exe):
    """The same scenario planned twice launches the same task arrays."""
    a = run(scenario_exe, *SCENARIOS["poisson3d_32_rank30"])
    b = run(scenario_exe, *SCENARIOS["poisson3d_32_rank30"])
    assert a["digest"] == b["digest"] and a["gemm_tiles"] == b["gemm_tiles"] and a["emu_tiles"] == b["emu_tiles"]
