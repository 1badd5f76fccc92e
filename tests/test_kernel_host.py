"""Host builds of branch_tron helpers whose exactness the kernel relies on.

The kernel's integer-pipe shortcuts and its bisected Cholesky shift are
claimed to give the same values as the plain operations: multiplications by
powers of two as exponent steps, and the first successful shift of the
Lin-More schedule found by bisection instead of in order.  These functions are
taken verbatim from the CUDA source, compiled for the host with g++ (CUDA
intrinsics replaced by bit casts) and checked against the plain computations
on random inputs.  No GPU is needed.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "..", "paper_2110_06879_gb300", "csrc", "branch_tron.cu")

SHIMS = r"""
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <random>
namespace K {
constexpr int kBranchBlock = 1;
constexpr int kCholTries = 20;
constexpr unsigned kFull = 0xffffffffu;
inline long long dbits(double v) { long long b; std::memcpy(&b, &v, 8); return b; }
inline double bitsd(long long b) { double v; std::memcpy(&v, &b, 8); return v; }
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
inline bool __any_sync(unsigned, bool p) { return p; }
"""

MAIN = r"""
// the schedule tried in order, as the oracle does
static int first_in_order(SMat H, const double *ds, const bool *fr, bool pos)
{
    double sigma = pos ? 0.0 : 1e-3, lb[32];
    SMat L{lb};
    for (int t = 0; t < kCholTries; ++t) {
        if (chol_pass<false>(H, ds, fr, sigma, true, L)) return t;
        sigma = std::max(sigma * 2.0, 1e-3);
    }
    return kCholTries;
}
}  // namespace K

int main()
{
    using namespace K;
    std::mt19937_64 rng(7);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    std::normal_distribution<double> N(0.0, 1.0);
    int bad = 0;
    // exponent steps against multiplication by powers of two
    for (int t = 0; t < 200000; ++t) {
        const double v = std::ldexp(U(rng), (int)(rng() % 600) - 300);
        const int k = (int)(rng() % 8);
        if (pow2_scale(v, k) != std::ldexp(v, -k)) ++bad;
        if (pow2_up(v, k) != std::ldexp(v, k)) ++bad;
        if (twice(v) != 2.0 * v) ++bad;
    }
    if (pow2_scale(0.0, 3) != 0.0 || pow2_up(0.0, 3) != 0.0 || twice(0.0) != 0.0) ++bad;
    for (int k = 0; k < kCholTries; ++k) {
        double s = 1e-3;
        for (int j = 0; j < k; ++j) s = std::max(s * 2.0, 1e-3);
        if (shift_at(k, false) != s) ++bad;
        if (shift_at(k + 1, true) != s) ++bad;
    }
    if (shift_at(0, true) != 0.0) ++bad;
    std::printf("exponent steps: %d mismatches\n", bad);
    // bisected shift against the schedule tried in order, on indefinite blocks
    int tested = 0, differ = 0;
    for (int t = 0; t < 40000; ++t) {
        double Q[6][6], ev[6], hb[32], lb[32], ls[32], db[32];
        for (int i = 0; i < 6; ++i)
            for (int j = 0; j < 6; ++j) Q[i][j] = N(rng);
        for (int i = 0; i < 6; ++i) ev[i] = std::exp(3.0 * N(rng)) * (rng() % 3 == 0 ? -1.0 : 1.0);
        SMat H{hb}, L{lb}, LS{ls}, D{db};
        for (int i = 0; i < 6; ++i)
            for (int j = i; j < 6; ++j) {
                double a = 0.0;
                for (int q = 0; q < 6; ++q) a += Q[i][q] * ev[q] * Q[j][q];
                H[P(i, j)] = a;
            }
        bool fr[6];
        unsigned frm = 0;
        for (int i = 0; i < 6; ++i) {
            fr[i] = rng() % 5 != 0;
            frm |= fr[i] ? 1u << i : 0u;
        }
        if (chol_pass<true>(H, nullptr, fr, 0.0, true, L)) continue;   // positive definite
        precond_scaled(true, H, frm, L, D);
        bool pos = true;
        double ds[6];
        for (int i = 0; i < 6; ++i) {
            const double a = H[P(i, i)];
            ds[i] = (fr[i] && okey(a) != 0) ? rsqrt(dabsi(a)) : 1.0;
            pos = pos && (!fr[i] || dpos(a));
        }
        const int k = first_in_order(H, ds, fr, pos);
        if (k < kCholTries) {
            chol_pass<false>(H, ds, fr, shift_at(k, pos), true, LS);
        } else {
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j <= i; ++j) LS[P(i, j)] = i == j ? 1.0 : 0.0;
        }
        ++tested;
        for (int q = 0; q < 21; ++q)
            if (L[q] != LS[q]) { ++differ; break; }
    }
    std::printf("bisected shift: %d blocks, %d different factors\n", tested, differ);
    return (bad == 0 && differ == 0 && tested > 10000) ? 0 : 1;
}
"""


def _between(text, start, end):
    i = text.index(start)
    return text[i:text.index(end, i)]


def _harness():
    src = open(SRC, encoding="utf-8").read()
    parts = [
        _between(src, "// packed symmetric index", "struct Cnt {"),
        _between(src, "// Order-preserving integer images of doubles", "// Two lanes per branch (kL = 2)"),
        _between(src, "// One Cholesky pass of M + sigma I", "// Returns whether the lane's factor"),
    ]
    code = SHIMS + "".join(parts) + MAIN
    for a, b in (("__host__ __device__ constexpr", "constexpr"), ("__device__ __forceinline__", "inline"),
                 ("__device__ __noinline__", "inline"), ("__double_as_longlong", "dbits"),
                 ("__longlong_as_double", "bitsd")):
        code = code.replace(a, b)
    return code


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_integer_steps_and_bisected_shift(tmp_path):
    cpp = tmp_path / "kernel_host.cpp"
    exe = tmp_path / "kernel_host"
    cpp.write_text(_harness())
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe), str(cpp)],
                   check=True, capture_output=True, text=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
