"""Pin of the oracle's Philox4x32-10 (the free-transport-time generator)
against an independent implementation: cuRAND's device Philox4x32-10, called
from a small CUDA program built for this test."""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

SRC = r"""
#include <cstdio>
#include <curand_kernel.h>
__global__ void k(const uint4* c, const uint2* key, uint4* out, int n) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = curand_Philox4x32_10(c[i], key[i]);
}
int main() {
    const int n = 512;
    uint4 hc[n]; uint2 hk[n]; uint4 ho[n];
    unsigned s = 12345u;
    for (int i = 0; i < n; ++i) {
        unsigned v[6];
        for (int j = 0; j < 6; ++j) { s = s * 1664525u + 1013904223u; v[j] = s; }
        if (i == 0) for (int j = 0; j < 6; ++j) v[j] = 0u;
        if (i == 1) for (int j = 0; j < 6; ++j) v[j] = 0xffffffffu;
        hc[i] = make_uint4(v[0], v[1], v[2], v[3]);
        hk[i] = make_uint2(v[4], v[5]);
    }
    uint4 *dc; uint2 *dk; uint4 *dout;
    cudaMalloc(&dc, sizeof(hc)); cudaMalloc(&dk, sizeof(hk)); cudaMalloc(&dout, sizeof(ho));
    cudaMemcpy(dc, hc, sizeof(hc), cudaMemcpyHostToDevice);
    cudaMemcpy(dk, hk, sizeof(hk), cudaMemcpyHostToDevice);
    k<<<(n + 127) / 128, 128>>>(dc, dk, dout, n);
    if (cudaMemcpy(ho, dout, sizeof(ho), cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
    for (int i = 0; i < n; ++i)
        printf("%u %u %u %u %u %u %u %u %u %u\n", hc[i].x, hc[i].y, hc[i].z, hc[i].w, hk[i].x, hk[i].y,
               ho[i].x, ho[i].y, ho[i].z, ho[i].w);
    return 0;
}
"""


def test_philox32_matches_curand():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "p.cu")
        exe = os.path.join(d, "p")
        with open(src, "w") as f:
            f.write(SRC)
        subprocess.run([nvcc, "-O2", "-gencode=arch=compute_103a,code=sm_103a", src, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = np.array([[int(v) for v in line.split()] for line in out.splitlines()], dtype=np.uint64)
    assert rows.shape == (512, 10)
    for r in rows:
        got = oracle.philox32(r[0:4].astype(np.uint32), r[4:6].astype(np.uint32))
        assert np.array_equal(got.astype(np.uint64), r[6:10])
