"""The device Philox4x32-10 generator against the oracle's CPU implementation and against cuRAND's
counter-based Philox4x32-10 (curand_Philox4x32_10 from curand_philox4x32_x.h), bit for bit."""
import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import oracle
from paper_2006_06775_gb300 import bdm
from paper_2006_06775_gb300 import build as libbuild

pytestmark = pytest.mark.gpu

CURAND_SRC = r"""
#include <curand_philox4x32_x.h>
#include <cuda_runtime.h>
__global__ void k(unsigned n, const uint4* c, const uint2* k, uint4* o) {
  unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) o[i] = curand_Philox4x32_10(c[i], k[i]);
}
extern "C" int curand_philox(unsigned n, const unsigned* c, const unsigned* key, unsigned* out) {
  void *dc, *dk, *dout;
  if (cudaMalloc(&dc, n * 16) || cudaMalloc(&dk, n * 8) || cudaMalloc(&dout, n * 16)) return 1;
  cudaMemcpy(dc, c, n * 16, cudaMemcpyHostToDevice);
  cudaMemcpy(dk, key, n * 8, cudaMemcpyHostToDevice);
  k<<<(n + 255) / 256, 256>>>(n, (const uint4*)dc, (const uint2*)dk, (uint4*)dout);
  int rc = cudaMemcpy(out, dout, n * 16, cudaMemcpyDeviceToHost) != cudaSuccess;
  cudaFree(dc); cudaFree(dk); cudaFree(dout);
  return rc;
}
"""


@pytest.fixture(scope="module")
def counters():
    g = np.random.default_rng(81)
    n = 1 << 16
    ctr = g.integers(0, 2 ** 32, (n, 4), dtype=np.uint64).astype(np.uint32)
    key = g.integers(0, 2 ** 32, (n, 2), dtype=np.uint64).astype(np.uint32)
    ctr[:4] = 0
    key[:2] = 0
    ctr[4:8] = 0xFFFFFFFF
    return ctr, key


def test_device_philox_matches_oracle(counters):
    ctr, key = counters
    assert np.array_equal(bdm.bdm_philox(ctr, key), oracle.philox(ctr, key))


def test_device_philox_matches_curand(counters):
    ctr, key = counters
    d = tempfile.mkdtemp()
    src = os.path.join(d, "curand_philox.cu")
    lib = os.path.join(d, "libcurand_philox.so")
    open(src, "w").write(CURAND_SRC)
    subprocess.run([libbuild.nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-shared",
                    "-Xcompiler", "-fPIC", src, "-o", lib], check=True)
    L = ctypes.CDLL(lib)
    out = np.zeros_like(ctr)
    assert L.curand_philox(len(ctr), ctr.ctypes.data_as(ctypes.c_void_p),
                           key.ctypes.data_as(ctypes.c_void_p),
                           out.ctypes.data_as(ctypes.c_void_p)) == 0
    assert np.array_equal(bdm.bdm_philox(ctr, key), out)
    assert np.array_equal(oracle.philox(ctr, key), out)
