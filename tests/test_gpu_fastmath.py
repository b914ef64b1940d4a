"""The FP64 step's reciprocal and reciprocal square root against correctly rounded values.

The FP64 kernels form 1/x and 1/sqrt(x) (and sqrt(x) = x / sqrt(x)) from the hardware
approximations refined by two Newton-Raphson steps, instead of IEEE division and square
root.  This test runs those device functions themselves (compiled here into a small probe
library from the kernel header) over the ranges the step feeds them: densities in
(0, 1/b), temperatures around the reduced range of the channels, the pseudopotential's
radicands, and a log-uniform sweep over twenty decades; and checks each result against
the correctly rounded value from a wider host format, in units in the last place.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2009_05264_gb300", "csrc")

PROBE = r'''
#include "lbm_kernels.cuh"
__global__ void probe(const double* x, double* r, double* q, double* s, long long n) {
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
    r[k] = pplbm::fast_rcp(x[k]);
    q[k] = pplbm::fast_rsqrt(x[k]);
    s[k] = pplbm::fast_sqrt(x[k]);
  }
}
extern "C" int run_probe(const double* x, double* r, double* q, double* s, long long n) {
  probe<<<152 * 4, 256>>>(x, r, q, s, n);
  return (int)cudaDeviceSynchronize();
}
'''


@pytest.fixture(scope="module")
def probe_lib(tmp_path_factory):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tmp_path_factory.mktemp("fastmath")
    src, lib = os.path.join(d, "probe.cu"), os.path.join(d, "libprobe.so")
    open(src, "w").write(PROBE)
    subprocess.check_call([nvcc, "-shared", "-Xcompiler", "-fPIC", "-O3", "-std=c++17", "-gencode",
                           "arch=compute_103a,code=sm_103a", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                           "-o", lib, src])
    L = ctypes.CDLL(lib)
    p = ctypes.c_void_p
    L.run_probe.argtypes = [p, p, p, p, ctypes.c_longlong]
    L.run_probe.restype = ctypes.c_int
    return L


def ulp_error(got, exact):
    """|got - exact| in units in the last place of the correctly rounded value."""
    ref = exact.astype(np.float64)
    return np.abs(got.astype(np.longdouble) - exact) / np.spacing(np.abs(ref)).astype(np.longdouble)


def inputs():
    rng = np.random.default_rng(2009052648)
    b = 2.0 / 21.0
    Tc = 0.0778 * (2.0 / 49.0) / (0.45724 * b)
    parts = [
        rng.uniform(1e-3, 1.0 / b, 200000),          # densities of the step, up to 1/b
        rng.uniform(0.3 * Tc, 2.0 * Tc, 200000),      # temperatures
        rng.uniform(1e-10, 20.0, 200000),             # psi radicands and 1 - b rho, 1 + 2 b rho - (b rho)^2
        10.0 ** rng.uniform(-10.0, 10.0, 200000),     # twenty decades
        np.array([1.0, 2.0, 4.0, 0.5, 1.0 / b - 1e-9, 1e-300 * 1e290]),
    ]
    return np.concatenate(parts)


def test_fp64_reciprocal_and_rsqrt_are_within_two_ulp(probe_lib):
    x = inputs()
    dev = torch.device("cuda", 0)
    tx = torch.from_numpy(x).to(dev)
    outs = [torch.empty_like(tx) for _ in range(3)]
    assert probe_lib.run_probe(*[ctypes.c_void_p(t.data_ptr()) for t in [tx] + outs], x.size) == 0
    r, q, s = (o.cpu().numpy() for o in outs)
    xl = x.astype(np.longdouble)
    e_r = ulp_error(r, 1.0 / xl)
    e_q = ulp_error(q, 1.0 / np.sqrt(xl))
    e_s = ulp_error(s, np.sqrt(xl))
    print(f"max ulp error: rcp {e_r.max():.3f}, rsqrt {e_q.max():.3f}, sqrt {e_s.max():.3f} "
          f"(long double epsilon {np.finfo(np.longdouble).eps:.1e})")
    if np.finfo(np.longdouble).eps >= np.finfo(np.float64).eps:
        pytest.skip("the host has no wider floating-point format than double for the reference")
    assert e_r.max() <= 2.0
    assert e_q.max() <= 2.0
    assert e_s.max() <= 2.5  # x times the refined rsqrt: one more rounding
    # against IEEE double division, which rounds correctly: the same to 2 ulp node by node
    assert np.all(np.abs(r - 1.0 / x) <= 2.0 * np.spacing(np.abs(1.0 / x)))
