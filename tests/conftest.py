import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def orc():
    import oracle
    oracle.build()
    return oracle


# Host emulations of the kernels (tests/host/*.cpp), compiled once per session
# and all at once: AddressSanitizer builds of the CTA emulation (one per shape),
# the persistent mesh kernel (per dimension and precision), the
# threading-over-elements kernel (per shape), the CG vector kernels and the
# geometric-factor kernel.
CSRC = os.path.join(ROOT, "paper_2606_20917_gb300", "csrc")
CUDA = "/usr/local/cuda"
HOST_BUILDS = {}
for _name, _sh in (("quad", 0), ("tri", 1), ("hex", 2), ("prism", 3), ("tet", 4), ("pyr", 5)):
    HOST_BUILDS[("cta", _name)] = ("cta_sim.cpp", ["-DSIM_HIGH_P", f"-DSIM_SHAPE={_sh}"], [])
    if _name != "pyr":
        HOST_BUILDS[("toe", _name)] = ("toe_sim.cpp", [f"-DSIM_SHAPE={_sh}"], [])
HOST_BUILDS[("cg",)] = ("cg_sim.cpp", ["-ffp-contract=off"], ["-L", os.path.join(CUDA, "lib64"), "-lcudart"])
HOST_BUILDS[("geom",)] = ("geom_sim.cpp", [], [])
for _dim, _prec, _code in ((3, "f32", 1), (2, "bf16", 2)):
    HOST_BUILDS[("mesh", _dim, _prec)] = ("mesh_sim.cpp", [f"-DNIR_MESH_DIM={_dim}", f"-DNIR_PREC={_code}"],
                                          ["-L", os.path.join(CUDA, "lib64"), "-lcudart"])


@pytest.fixture(scope="session")
def host_sims(tmp_path_factory):
    """{key: executable} for every entry of HOST_BUILDS."""
    gxx = shutil.which("g++")
    if not gxx or not os.path.isdir(os.path.join(CUDA, "include")):
        pytest.skip("g++ or the CUDA headers are not available")
    out = tmp_path_factory.mktemp("host_sims")

    def build(key):
        src, defs, libs = HOST_BUILDS[key]
        exe = str(out / "_".join(str(k) for k in key))
        cmd = [gxx, "-O0", "-g1", "-std=c++17", "-w", "-fno-omit-frame-pointer", "-fsanitize=address", *defs,
               "-I", os.path.join(CUDA, "include"), "-I", CSRC, "-I", os.path.join(ROOT, "include"),
               os.path.join(ROOT, "tests", "host", src), os.path.join(CSRC, "nir_basis.cpp"), "-o", exe,
               *libs, "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, (key, r.stderr[-3000:])
        return key, exe

    # the slowest builds first
    keys = sorted(HOST_BUILDS, key=lambda k: {"cta": 0, "mesh": 1, "toe": 2, "cg": 3, "geom": 4}[k[0]])
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        return dict(ex.map(build, keys))
