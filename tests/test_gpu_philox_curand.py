"""Philox4x32-10 against NVIDIA's own implementation: cuRAND's device API
(curand_init + curand4 on curandStatePhilox4_32_10_t).  cuRAND keys the
generator with the 64-bit seed and keeps a 128-bit counter whose low 64 bits
advance by offset / 4 (skipahead) and whose high 64 bits advance by the
subsequence, so counter (g, lattice, t, c) is subsequence t + 2^32 c at offset
4 (g + 2^32 lattice).  The oracle's generator, which the sweeps' random numbers
match bit for bit, must equal it on a spread of counters and keys."""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SRC = r'''
#include <curand_kernel.h>
__global__ void draws(const unsigned long long *seed, const unsigned long long *subseq,
                      const unsigned long long *offset, uint4 *out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    curandStatePhilox4_32_10_t st;
    curand_init(seed[i], subseq[i], offset[i], &st);
    out[i] = curand4(&st);
}
extern "C" int run_draws(const unsigned long long *seed, const unsigned long long *subseq,
                         const unsigned long long *offset, unsigned int *out, int n) {
    unsigned long long *d_seed, *d_sub, *d_off; uint4 *d_out;
    size_t b = sizeof(unsigned long long) * n;
    cudaMalloc(&d_seed, b); cudaMalloc(&d_sub, b); cudaMalloc(&d_off, b); cudaMalloc(&d_out, 16 * (size_t)n);
    cudaMemcpy(d_seed, seed, b, cudaMemcpyHostToDevice);
    cudaMemcpy(d_sub, subseq, b, cudaMemcpyHostToDevice);
    cudaMemcpy(d_off, offset, b, cudaMemcpyHostToDevice);
    draws<<<(n + 127) / 128, 128>>>(d_seed, d_sub, d_off, d_out, n);
    cudaError_t e = cudaMemcpy(out, d_out, 16 * (size_t)n, cudaMemcpyDeviceToHost);
    cudaFree(d_seed); cudaFree(d_sub); cudaFree(d_off); cudaFree(d_out);
    return (int)e;
}
'''


@pytest.fixture(scope="module")
def curand_lib(tmp_path_factory):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    d = tmp_path_factory.mktemp("curand")
    src, so = d / "draws.cu", d / "draws.so"
    src.write_text(SRC)
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-shared",
                           "-Xcompiler", "-fPIC", str(src), "-o", str(so)])
    lib = ctypes.CDLL(str(so))
    p64 = ctypes.POINTER(ctypes.c_ulonglong)
    lib.run_draws.argtypes = [p64, p64, p64, ctypes.POINTER(ctypes.c_uint), ctypes.c_int]
    return lib


def test_oracle_philox_equals_curand(curand_lib):
    rng = np.random.default_rng(12)
    n = 4096
    g = rng.integers(0, 2 ** 32, n, dtype=np.uint64)
    lat = rng.integers(0, 2 ** 30, n, dtype=np.uint64)     # offset 4 (g + 2^32 lattice) < 2^64
    t = rng.integers(0, 2 ** 32, n, dtype=np.uint64)
    c = rng.integers(0, 4, n, dtype=np.uint64)
    seed = rng.integers(0, 2 ** 63, n, dtype=np.uint64)
    g[:4], lat[:4], t[:4], c[:4] = 0, 0, 0, 0
    t[4:8] = 0xFFFFFFFF                          # the initialisation counters
    subseq = (t | (c << np.uint64(32))).astype(np.uint64)
    offset = (np.uint64(4) * (g | (lat << np.uint64(32)))).astype(np.uint64)
    out = np.zeros((n, 4), dtype=np.uint32)
    p64 = ctypes.POINTER(ctypes.c_ulonglong)
    rc = curand_lib.run_draws(seed.ctypes.data_as(p64), subseq.ctypes.data_as(p64), offset.ctypes.data_as(p64),
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint)), n)
    assert rc == 0
    for i in range(n):
        key = [int(seed[i]) & 0xFFFFFFFF, int(seed[i]) >> 32]
        want = oracle.philox4x32_10([int(g[i]), int(lat[i]), int(t[i]), int(c[i])], key)
        assert np.array_equal(out[i], want), i


@pytest.mark.parametrize("g0,n", [(0, 1), (12345, 100003), (2**32 - 4099, 4099), (7, 0)])
def test_philox_stream_digest_matches_the_oracle(g0, n):
    """The library's stream code (the sweeps' Philox path with its hoisted
    products) against the oracle's Philox, through a digest of every word."""
    import paper_2304_01772_gb300 as sm
    seed, lat, t, c = 0xFEEDFACE12345678, 300, 4242, 1
    got = int(sm.philox_xor(seed, lat, t, c, g0, n).cpu().numpy().view(np.uint32)[0])
    assert got == oracle.philox_xor(seed, lat, t, c, g0, n)


def test_philox_stream_digest_rejects_ranges_past_the_counter():
    import paper_2304_01772_gb300 as sm
    with pytest.raises(sm.SpinError):
        sm.philox_xor(1, 0, 0, 0, 2**32 - 10, 11)
