"""Host logic of the chunk layout (ChunkLayout in csrc/rt_kernels.cuh), compiled for the CPU with
nvcc and run there: it splits the rays of a longest-first order into chunks for the overlapped
shapes, and places each rank of the sort. For many (n, K, W):
- the chunk sizes sum to n, the offsets are their prefix sums, and max_size is the largest;
- place() is a bijection of the ranks onto [0, n);
- each chunk receives its ranks in increasing order (so each chunk runs longest first), and the
  ranks are dealt in rounds of (K - 1) W + 1: W to each regular chunk in turn, one to the last;
- chunk_of() returns the chunk whose range holds an index;
- with W = 1 the layout is the round-robin one: chunk k holds n / K + (k < n % K) rays from
  k (n / K) + min(k, n % K), rank s going to chunk s % K.
No GPU is used."""
import os
import subprocess
import tempfile

import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)

SRC = r"""
#include <cstdio>
#include <vector>
#include <algorithm>
#include "rt_kernels.cuh"
using prt::ChunkLayout;
static int fail(const char *what, long long n, int K, int W, long long x) {
    std::printf("FAIL %s n=%lld K=%d W=%d at %lld\n", what, n, K, W, x);
    return 1;
}
int check(long long n, int K, int W) {
    ChunkLayout L{n, K, W};
    long long sum = 0, mx = 0;
    for (int k = 0; k < K; k++) {
        if (L.offset(k) != sum) return fail("offset", n, K, W, k);
        if (L.size(k) < 0) return fail("size", n, K, W, k);
        sum += L.size(k);
        mx = std::max(mx, L.size(k));
    }
    if (sum != n) return fail("sum", n, K, W, sum);
    if (L.max_size() != mx) return fail("max_size", n, K, W, mx);
    std::vector<char> seen(n, 0);
    std::vector<long long> last(K, -1);
    const long long P = (long long)(K - 1) * W + 1;
    for (long long s = 0; s < n; s++) {
        long long t = L.place(s);
        if (t < 0 || t >= n || seen[t]) return fail("place", n, K, W, s);
        seen[t] = 1;
        int k = L.chunk_of(t);
        if (t < L.offset(k) || t >= L.offset(k) + L.size(k)) return fail("chunk_of", n, K, W, t);
        if (t <= last[k]) return fail("order", n, K, W, s);
        last[k] = t;
        long long j = s % P;
        int want = j < (long long)(K - 1) * W ? (int)(j / W) : K - 1;
        if (k != want) return fail("deal", n, K, W, s);
        if (W == 1) {
            long long b = n / K, e = n % K;
            if (t != (s % K) * b + std::min<long long>(s % K, e) + s / K) return fail("round-robin", n, K, W, s);
        }
    }
    return 0;
}
int main() {
    int bad = 0, cases = 0;
    const long long ns[] = {1, 2, 3, 7, 31, 32, 33, 100, 255, 1000, 4097, 12345, 65536};
    const int Ks[] = {1, 2, 3, 4, 7, 8, 16, 33, 64};
    const int Ws[] = {1, 2, 3, 4, 16};
    for (long long n : ns)
        for (int K : Ks)
            for (int W : Ws) {
                if (K > n) continue;
                bad += check(n, K, W);
                cases++;
            }
    std::printf("cases %d failures %d\n", cases, bad);
    return bad != 0;
}
"""


def test_chunk_layout_host_logic():
    from paper_2302_02733_gb300 import build

    try:
        nvcc = build.nvcc()
    except RuntimeError:
        pytest.skip("no nvcc")
    csrc = os.path.join(__graft_entry__.ROOT, "paper_2302_02733_gb300", "csrc")
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.cu"), os.path.join(d, "layout")
        with open(src, "w") as f:
            f.write(SRC)
        r = subprocess.run([nvcc, "-std=c++17", "-O1", "-I", csrc, "-o", exe, src], capture_output=True, text=True)
        assert r.returncode == 0, r.stderr
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stdout + r.stderr
        assert "failures 0" in r.stdout
