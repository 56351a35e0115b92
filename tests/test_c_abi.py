"""The library used from plain C: tests/c_abi/abi_client.c is compiled with gcc
against include/pmf.h alone and linked with libpmf.so (no Python, no torch in
that process).  The host-only calls run without a GPU; the solves (through a
batch and through pmf_solve_noalloc) run on the GPU and are compared with the
oracle element by element."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1509_06004_b300 import build as pbuild
from paper_1509_06004_b300 import inputs, pmf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


@pytest.fixture(scope="module")
def client(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    pbuild.build()
    libdir = os.path.dirname(pmf.LIB_PATH)
    exe = str(tmp_path_factory.mktemp("c_abi") / "abi_client")
    subprocess.check_call([
        "gcc", "-O2", "-std=c11", "-Wall", "-Wextra", "-Werror",
        "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(CUDA, "include"),
        os.path.join(ROOT, "tests", "c_abi", "abi_client.c"),
        "-L" + libdir, "-lpmf", "-Wl,-rpath," + libdir,
        "-L" + os.path.join(CUDA, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(CUDA, "lib64"),
        "-o", exe])
    return exe


def test_header_compiles_as_strict_c_and_cxx(tmp_path):
    """The header alone builds in strict C and in C++ (extern "C" guards)."""
    src = tmp_path / "h.c"
    src.write_text('#include "pmf.h"\nint main(void) { return pmf_version() == 0; }\n')
    inc = "-I" + os.path.join(ROOT, "include")
    subprocess.check_call(["gcc", "-std=c99", "-pedantic", "-Wall", "-Werror", inc, "-c", str(src),
                           "-o", str(tmp_path / "h.o")])
    subprocess.check_call(["g++", "-std=c++17", "-Wall", "-Werror", inc, "-x", "c++", "-c", str(src),
                           "-o", str(tmp_path / "hpp.o")])


def test_host_calls_from_c(client):
    r = subprocess.run([client, "host"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    _, _, a, b = r.stdout.split()
    assert int(a) == pmf.workspace_size([(64, 64), (240, 320)], [0, 1, 1], 20)
    assert int(b) == pmf.workspace_size([(64, 64), (240, 320)], [0, 1, 1], 40)


def write_problem(path, H, W, lambdas, w_h, w_v, src0, slope, sink):
    with open(path, "wb") as f:
        np.array([H, W, len(lambdas)], "<i4").tofile(f)
        np.asarray(lambdas, "<i4").tofile(f)
        for a in (w_h, w_v, src0, slope, sink):
            np.ascontiguousarray(a, "<i4").reshape(H, W).tofile(f)


def read_result(path, H, W, m):
    raw = open(path, "rb").read()
    flows = np.frombuffer(raw[:8 * m], "<i8")
    masks = np.frombuffer(raw[8 * m:], np.uint8).reshape(m, H, W)
    return flows, masks


def problem(H, W, seed):
    """A segmentation instance of the paper's form: contrast-sensitive
    pairwise capacities of a synthetic image, a seed square's terminals and
    an increasing lambda schedule."""
    rng = np.random.default_rng(seed)
    img = inputs.make_image(H, W, 4, 0.05, rng)
    w_h, w_v = inputs.pairwise_caps(img)
    y0, x0 = inputs.random_seed_origin(H, W, rng)
    src0, slope, sink = inputs.terminals(img, inputs.seed_square(H, W, y0, x0))
    lam = inputs.lambda_schedule(6, 10, 5000)
    return w_h, w_v, src0, slope, sink, lam


@pytest.mark.gpu
@pytest.mark.parametrize("mode", ["solve", "noalloc", "server"])
@pytest.mark.parametrize("shape", [(37, 45), (70, 90)])
def test_solve_from_c_matches_oracle(client, tmp_path, mode, shape):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    H, W = shape
    w_h, w_v, src0, slope, sink, lam = problem(H, W, H * 7 + W)
    write_problem(tmp_path / "in.bin", H, W, lam, w_h, w_v, src0, slope, sink)
    r = subprocess.run([client, mode, str(tmp_path / "in.bin"), str(tmp_path / "out.bin")],
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    flows, masks = read_result(tmp_path / "out.bin", H, W, len(lam))
    of, om = oracle.grid_solve(H, W, w_h, w_v, src0, slope, sink, lam)
    assert np.array_equal(flows, of), (flows, of)
    assert np.array_equal(masks, om), np.argwhere(masks != om)[:10]
