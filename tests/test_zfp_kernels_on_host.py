"""The fixed-rate ZFP kernels' own code, built for the host, against the
oracle (CPU only).

The encoder and decoder kernels of csrc/zfp.cu use nothing but integer and
double arithmetic plus four CUDA built-ins (__ffs, __ffsll, __double2ll_rz and
the thread indices), so the same source compiles as host C++ with those
defined.  One "thread" per block then walks every block of a field, and the
words and values must equal the oracle's bit for bit: a check of the kernel
logic that needs no GPU (the GPU tests check the same on the device)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_2503_06322_gb300", "csrc", "zfp.cu")

PRELUDE = r'''
#include <cstdint>
#include <cstring>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>
#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __launch_bounds__(x)
struct U3 { unsigned x; };
static U3 blockIdx, threadIdx, blockDim;
static inline int __ffs(int x) { return __builtin_ffs(x); }
static inline int __ffsll(long long x) { return __builtin_ffsll(x); }
static inline long long __double2ll_rz(double x) { return (long long)x; }
namespace hz {
'''

MAIN = r'''
}
using namespace hz;
template <typename T, int D> void run(const char *fin, const char *fw, const char *fwin, const char *fout,
                                      long long N, ZfpGeom g)
{
    std::vector<T> in(N), out(N);
    FILE *f = fopen(fin, "rb"); if (fread(in.data(), sizeof(T), N, f) != (size_t)N) exit(2); fclose(f);
    std::vector<uint32_t> w(g.nblocks * (g.maxbits / 32), 0xDEADBEEFu), w2(w.size());
    blockDim.x = 1; threadIdx.x = 0;
    for (unsigned long long b = 0; b < g.nblocks; b++) { blockIdx.x = (unsigned)b; zfp_encode_kernel<T, D>(in.data(), w.data(), g); }
    f = fopen(fw, "wb"); fwrite(w.data(), 4, w.size(), f); fclose(f);
    f = fopen(fwin, "rb"); if (fread(w2.data(), 4, w2.size(), f) != w2.size()) exit(3); fclose(f);
    for (unsigned long long b = 0; b < g.nblocks; b++) { blockIdx.x = (unsigned)b; zfp_decode_kernel<T, D>(w2.data(), out.data(), g); }
    f = fopen(fout, "wb"); fwrite(out.data(), sizeof(T), N, f); fclose(f);
}
int main(int argc, char **argv)
{
    int dtype = atoi(argv[5]), nd = atoi(argv[6]);
    long long n[3] = {atoll(argv[7]), atoll(argv[8]), atoll(argv[9])};
    unsigned rate = (unsigned)atoi(argv[10]);
    ZfpGeom g; memset(&g, 0, sizeof(g)); g.nblocks = 1;
    long long N = 1;
    for (int k = 0; k < 3; k++) {
        g.n[k] = k < nd ? n[k] : 1; g.nb[k] = (g.n[k] + 3) / 4;
        if (k < nd) { g.nblocks *= g.nb[k]; N *= n[k]; }
    }
    g.maxbits = rate << (2 * nd);
    if (dtype == 0) {
        if (nd == 1) run<float, 1>(argv[1], argv[2], argv[3], argv[4], N, g);
        else if (nd == 2) run<float, 2>(argv[1], argv[2], argv[3], argv[4], N, g);
        else run<float, 3>(argv[1], argv[2], argv[3], argv[4], N, g);
    } else {
        if (nd == 1) run<double, 1>(argv[1], argv[2], argv[3], argv[4], N, g);
        else if (nd == 2) run<double, 2>(argv[1], argv[2], argv[3], argv[4], N, g);
        else run<double, 3>(argv[1], argv[2], argv[3], argv[4], N, g);
    }
    return 0;
}
'''


@pytest.fixture(scope="module")
def host_exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = open(SRC).read()
    a = src.index("constexpr int kZfpThreads")
    b = src.index("__global__ void zfp_header_kernel")
    d = tmp_path_factory.mktemp("zfp_host")
    cpp = d / "zfp_host.cpp"
    cpp.write_text(PRELUDE + src[a:b] + MAIN)
    exe = d / "zfp_host"
    subprocess.run([cxx, "-O1", "-std=c++17", "-o", str(exe), str(cpp)], check=True)
    return str(exe), d


CASES = [((1000,), 8), ((7,), 32), ((65, 33), 2), ((9, 6), 12), ((33, 17, 9), 4), ((5, 6, 7), 16),
         ((4, 4, 4), 1), ((20, 30, 40), 136)]


@pytest.mark.parametrize("shape,rate", CASES, ids=str)
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_kernel_code_matches_oracle(host_exe, shape, rate, dtype):
    from paper_2503_06322_gb300 import fields
    exe, d = host_exe
    if len(shape) == 1:
        u = np.random.default_rng(5).standard_normal(shape).astype(dtype)
    else:
        u = fields.powerlaw_field(shape, seed=5, dtype=dtype)
    if len(shape) == 2:
        u[:4, :4] = 0.0
        u[4:8, :4] = 2.25
    ob = oracle.zfp_compress(u, rate)
    fin, fw, fwin, fout = (str(d / x) for x in ("in.bin", "w.bin", "win.bin", "out.bin"))
    np.ascontiguousarray(u).tofile(fin)
    ob[64:].tofile(fwin)
    n = list(shape) + [1] * (3 - len(shape))
    subprocess.run([exe, fin, fw, fwin, fout, "0" if dtype == np.float32 else "1", str(len(shape)),
                    *map(str, n), str(rate)], check=True)
    assert np.array_equal(np.fromfile(fw, dtype=np.uint8), ob[64:])
    assert np.array_equal(np.fromfile(fout, dtype=dtype).reshape(shape), oracle.zfp_decompress(ob).astype(dtype))
