"""The host preprocessing (cleaning, orderings, classifier, relabelling)
built with AddressSanitizer and UndefinedBehaviorSanitizer and driven over
awkward inputs: empty and one-vertex graphs, isolated vertices, duplicates,
self-loops, hub rows, windows larger than the graph, invalid CSR."""
import os
import shutil
import subprocess

import pytest

from conftest import ROOT

CSRC = os.path.join(ROOT, "paper_2512_21967_gb300", "csrc")
DRIVER = os.path.join(ROOT, "tests", "host", "sanitize_driver.cpp")


def test_host_preprocessing_under_asan_ubsan(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "sanitize_driver")
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fno-omit-frame-pointer", "-fsanitize=address,undefined",
           "-fno-sanitize-recover=undefined", "-I", CSRC, os.path.join(CSRC, "host_graph.cpp"), DRIVER,
           "-o", exe, "-pthread"]
    build = subprocess.run(cmd, capture_output=True, text=True)
    if build.returncode != 0 and "sanitize" in build.stderr and "cannot find" in build.stderr:
        pytest.skip("sanitizer runtime not installed")
    assert build.returncode == 0, build.stderr[-3000:]
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=1", UBSAN_OPTIONS="halt_on_error=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    assert run.returncode == 0, (run.stdout[-2000:], run.stderr[-4000:])
    assert "runtime error" not in run.stderr
    assert "failures=0" in run.stdout


def test_multi_source_chunk_sizing(tmp_path):
    """Every chunk the multi-source launcher makes fits the state a caller sizes
    for the whole launch with the same functions (the server's pre-allocation)."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    cuda_inc = None
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            cuda_inc = os.path.join(d, "include")
            break
    if cuda_inc is None:
        pytest.skip("no CUDA headers")
    exe = str(tmp_path / "msbfs_sizing")
    cmd = [gxx, "-std=c++17", "-O1", "-fsanitize=undefined", "-fno-sanitize-recover=undefined", "-I", CSRC,
           "-I", cuda_inc, os.path.join(ROOT, "tests", "host", "msbfs_sizing.cpp"), "-o", exe]
    build = subprocess.run(cmd, capture_output=True, text=True)
    if build.returncode != 0 and "sanitize" in build.stderr and "cannot find" in build.stderr:
        pytest.skip("sanitizer runtime not installed")
    assert build.returncode == 0, build.stderr[-3000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and "failures=0" in run.stdout, run.stdout[-2000:]


def test_msbfs_bit_plane_helpers(tmp_path):
    """The multi-source level bit planes: the 8 x 8 bit transpose and the
    per-source level extraction against their loop definitions, and the plane
    count against the largest level an n-vertex graph can have."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "msbfs_bits_check")
    cmd = [gxx, "-std=c++17", "-O1", "-fsanitize=undefined", "-fno-sanitize-recover=undefined", "-I", CSRC,
           os.path.join(ROOT, "tests", "host", "msbfs_bits_check.cpp"), "-o", exe]
    build = subprocess.run(cmd, capture_output=True, text=True)
    if build.returncode != 0 and "sanitize" in build.stderr and "cannot find" in build.stderr:
        pytest.skip("sanitizer runtime not installed")
    assert build.returncode == 0, build.stderr[-3000:]
    run = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert run.returncode == 0 and "failures=0" in run.stdout, run.stdout[-2000:]


def test_host_preprocessing_under_tsan(tmp_path):
    """The same driver built with ThreadSanitizer: the threaded parts (cleaning,
    symmetry check, relabelling, JaccardWithWindows, the parallel levels of the
    RCM pseudo-peripheral search) run without data races."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    exe = str(tmp_path / "sanitize_driver_tsan")
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fsanitize=thread", "-I", CSRC, os.path.join(CSRC, "host_graph.cpp"),
           DRIVER, "-o", exe, "-pthread"]
    build = subprocess.run(cmd, capture_output=True, text=True)
    if build.returncode != 0 and "sanitize" in build.stderr and "cannot find" in build.stderr:
        pytest.skip("sanitizer runtime not installed")
    assert build.returncode == 0, build.stderr[-3000:]
    env = dict(os.environ, TSAN_OPTIONS="halt_on_error=1")
    run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=600)
    if run.returncode != 0 and "unexpected memory mapping" in run.stderr:
        pytest.skip("ThreadSanitizer cannot run under this kernel's address layout")
    assert run.returncode == 0, (run.stdout[-2000:], run.stderr[-4000:])
    assert "ThreadSanitizer" not in run.stderr
    assert "failures=0" in run.stdout
