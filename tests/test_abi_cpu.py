"""The C-ABI library builds for sm_103a, loads, and exports every entry point
include/fire.h declares (no GPU needed: nothing is called)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fire.h")


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(
        r"^FIRE_API\s+(?:const\s+)?\w+\s*\**\s*(\w+)\s*\(", txt,
        flags=re.M)))


@pytest.fixture(scope="module")
def libpath():
    from paper_1701_03549_gb300 import build

    return build.build_library()


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("fire_create", "fire_maps_upload", "fire_target_upload",
                     "fire_simulate_batch", "fire_fitness", "ga_step"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    lib = ctypes.CDLL(libpath)
    for name in _declared():
        assert hasattr(lib, name), name


def test_only_abi_symbols_are_exported(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath],
                         capture_output=True, text=True, check=True).stdout
    text_syms = [l.split()[-1] for l in out.splitlines() if " T " in l]
    assert sorted(text_syms) == _declared()


def test_binding_covers_the_header():
    from paper_1701_03549_gb300 import fire

    assert sorted(fire.EXPORTED) == _declared()


def test_binding_loads_without_a_gpu(libpath):
    from paper_1701_03549_gb300 import fire

    L = fire.load()
    assert L.fire_simulate_batch.restype is ctypes.c_int


def test_missing_library_fails_loudly(tmp_path):
    from paper_1701_03549_gb300 import fire

    saved = fire._lib
    fire._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            fire.load(str(tmp_path / "libfire.so"))
    finally:
        fire._lib = saved


def test_kernels_compile_for_sm103a_with_little_spilling():
    from paper_1701_03549_gb300 import build

    src = os.path.join(build.CSRC, "fire_kernels.cu")
    r = subprocess.run([build._nvcc(), *build.ARCH, *build.NVCC_FLAGS,
                        "-Xptxas=-v", "-c", src, "-o", os.devnull],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    seen = 0
    for block in r.stderr.split("Compiling entry function")[1:]:
        if "k_simulate" in block.split("\n")[0]:
            seen += 1
            spill = int(re.search(r"(\d+) bytes spill stores", block).group(1))
            assert spill <= 64, block
    assert seen == 3    # shared / global state, and the burn-time variant


def test_tile_row_division_by_magic_multiply():
    """The simulation kernel finds a tile's row as (k + 1) * m >> 32 with
    m = floor((2^32 - 1) / TW); this equals k // TW for every tile index and
    every tile-grid width the library accepts (up to FIRE_MAX_TILES)."""
    import numpy as np

    hdr = open(HEADER).read()
    n = int(re.search(r"#define FIRE_MAX_TILES (\d+)", hdr).group(1))
    k = np.arange(n, dtype=np.uint64)[None, :]
    for lo in range(1, n + 1, 512):
        TW = np.arange(lo, min(lo + 512, n + 1), dtype=np.uint64)[:, None]
        m = np.uint64(2 ** 32 - 1) // TW
        q = ((k + np.uint64(1)) * m) >> np.uint64(32)
        assert np.array_equal(q, k // TW), lo


def test_simulation_guards_refuse_before_any_cuda_call(libpath, tmp_path):
    """A map uploaded on another device than the context's, and flags the
    no-alloc entry point does not honour, are refused with FIRE_EINVAL before
    any CUDA call: contexts and maps are built in host memory by a small
    program compiled against the library (tests/abi_guards_host.cu), so the
    checks run here without a GPU."""
    from paper_1701_03549_gb300 import build

    src = os.path.join(ROOT, "tests", "abi_guards_host.cu")
    so = str(tmp_path / "libabi_guards.so")
    libdir = os.path.dirname(libpath)
    cmd = [build._nvcc(), *build.ARCH, "-std=c++17", "-O1", "-Xcompiler",
           "-fPIC", "-shared", "-I", build.INCLUDE, "-I", build.CSRC, src,
           "-o", so, "-L" + libdir, "-lfire", "-Xlinker", "-rpath=" + libdir]
    subprocess.run(cmd, check=True, capture_output=True)
    lib = ctypes.CDLL(so)
    msg = ctypes.create_string_buffer(512)
    rc = lib.abi_guard_cases(msg, 512)
    assert rc == 0, msg.value.decode()


def _guards_lib(libpath, tmp_path):
    from paper_1701_03549_gb300 import build

    src = os.path.join(ROOT, "tests", "abi_guards_host.cu")
    so = str(tmp_path / "libabi_guards.so")
    libdir = os.path.dirname(libpath)
    subprocess.run([build._nvcc(), *build.ARCH, "-std=c++17", "-O1",
                    "-Xcompiler", "-fPIC", "-shared", "-I", build.INCLUDE,
                    "-I", build.CSRC, src, "-o", so, "-L" + libdir, "-lfire",
                    "-Xlinker", "-rpath=" + libdir],
                   check=True, capture_output=True)
    return so


def test_entry_points_open_nvtx_ranges(libpath, tmp_path):
    """Each C-ABI compute call opens an NVTX range named after itself and
    closes it on every return path: a minimal NVTX tool
    (tests/nvtx_capture.c, loaded through NVTX_INJECTION64_PATH) records the
    ranges of calls the argument guards refuse, in a child process without a
    GPU."""
    import sys

    from paper_1701_03549_gb300 import build

    guards = _guards_lib(libpath, tmp_path)
    tool = str(tmp_path / "libnvtx_capture.so")
    cuda_inc = os.path.join(os.path.dirname(os.path.dirname(build._nvcc())),
                            "include")
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-I", cuda_inc,
                    os.path.join(ROOT, "tests", "nvtx_capture.c"), "-o", tool],
                   check=True)
    child = (
        "import ctypes\n"
        f"tool = ctypes.CDLL({tool!r})\n"
        f"g = ctypes.CDLL({guards!r})\n"
        "msg = ctypes.create_string_buffer(512)\n"
        "assert g.abi_guard_cases(msg, 512) == 0, msg.value\n"
        "tool.nvtx_capture_names.restype = ctypes.c_char_p\n"
        "print(tool.nvtx_capture_names().decode().replace(chr(10), ' '))\n"
        "print(tool.nvtx_capture_depth())\n")
    env = dict(os.environ, NVTX_INJECTION64_PATH=tool)
    out = subprocess.run([sys.executable, "-c", child], env=env,
                         capture_output=True, text=True, check=True).stdout
    names, depth = out.strip().split("\n")
    assert "fire_simulate_batch" in names.split(), names
    assert int(depth) == 0
