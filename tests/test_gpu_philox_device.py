"""Counter word 3 of the oracle's Philox4x32-10, pinned against cuRAND's
device generator (an independent implementation, run, not copied).

curand_init(seed, subsequence, offset) starts the Philox counter at
(offset / 4 as a 64-bit value in words 0-1, subsequence in words 2-3) with
key (seed lo, seed hi), and the first curand4() returns that counter's four
output words.  Subsequences at and above 2^32 set word 3; offsets at and
above 2^34 set word 1.  A tiny kernel is compiled at test time with nvcc."""
import ctypes
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SRC = r'''
#include <cstdint>
#include <curand_kernel.h>
__global__ void draw(unsigned long long seed, unsigned long long subseq, unsigned long long offset, uint4* out)
{
    curandStatePhilox4_32_10_t s;
    curand_init(seed, subseq, offset, &s);
    *out = curand4(&s);
}
extern "C" int curand_device_quad(unsigned long long seed, unsigned long long subseq, unsigned long long offset,
                                  unsigned int* host)
{
    uint4* d = nullptr;
    if (cudaMalloc(&d, sizeof(uint4)) != cudaSuccess) return 1;
    draw<<<1, 1>>>(seed, subseq, offset, d);
    cudaError_t e = cudaMemcpy(host, d, sizeof(uint4), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : 2;
}
'''


@pytest.fixture(scope="module")
def curand_device():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("CUDA device required")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tempfile.mkdtemp()
    src = os.path.join(d, "draw.cu")
    lib = os.path.join(d, "libdraw.so")
    open(src, "w").write(SRC)
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", "-o", lib, src])
    so = ctypes.CDLL(lib)
    so.curand_device_quad.argtypes = [ctypes.c_ulonglong] * 3 + [ctypes.POINTER(ctypes.c_uint)]
    yield so
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("seed,subseq,quad", [
    (0x0123456789ABCDEF, 0, 0), (0x0123456789ABCDEF, 5, 7), (1, 2**32, 0), (1, 2**32 + 9, 3),
    (0xDEADBEEFCAFEF00D, 0xFFFFFFFFFFFFFFFF, 2**40 + 1), (2**64 - 1, 3 * 2**32 + 1, 2**33 + 5),
])
def test_philox_matches_curand_device(curand_device, oracle_lib, seed, subseq, quad):
    out = (ctypes.c_uint * 4)()
    assert curand_device.curand_device_quad(seed, subseq, 4 * quad, out) == 0
    ctr = (quad & 0xFFFFFFFF, quad >> 32, subseq & 0xFFFFFFFF, subseq >> 32)
    got = oracle_lib.philox4x32_10(ctr, (seed & 0xFFFFFFFF, seed >> 32))
    assert np.array_equal(got, np.frombuffer(out, dtype=np.uint32)), (hex(seed), hex(subseq), quad)
