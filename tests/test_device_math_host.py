"""The CUDA path's device arithmetic compiled for the host and checked against the oracle on the CPU.

The per-face and per-cell functions of mhd_device.cuh (PPM parabolas, the streamed parabolas, the
Riemann solve, the chemistry of one cell, the CFL denominator) are plain C++ apart from a block of
inline-PTX helpers (integer-pipe tests, the reciprocal and reciprocal-square-root seeds of the
Newton-Raphson forms); this test replaces that block with portable C++ of the same definitions, compiles tests/host_math/device_math_vs_oracle.cpp against it and the oracle library,
and checks: the FP64 parabolas are within 3e-15 of the stencil's largest value of the oracle's (Sec. 2.1;
q6 is formed as 6 q_c - 3 (q_L + q_R), and the Step 4 blend's eta takes the Newton-Raphson reciprocal), the
streamed ones equal the five-point ones bit for bit, so do the FP32 pencils' parabolas built from
carried slopes (ppm_carried against ppm_direct), the Riemann solve (Sec. 2.4, App. A) is within 1e-12 of the
oracle's in FP64 and 1e-4 in FP32, the chemistry (Sec. 2.7, App. D; with and without reactions 5-8)
within 1e-12, the heating/cooling change (Sec. 2.8; with and without Gamma_5 and Lambda_6-8) within
1e-12 of the gross heating plus cooling, the Newton-Raphson reciprocal, reciprocal square root
and square root within 2 ulp of the correctly rounded values, the CFL
denominator (Sec. 2.3) within 1e-13, the table-driven exponential of the chemistry within 1.01 ulp of
e^x (long-double reference), and the FP32 estimate of the CFL screen within 64 u (u = 2^-24) of the
FP64 denominator wherever its guards pass, on inputs over many decades, with and without the H/H2
mixture's gamma.  The host build uses -ffp-contract=off like the oracle; the
GPU build contracts to FMA, whose effect the GPU parity tests bound."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_1608_08748_gb300", "csrc", "mhd_device.cuh")
HARNESS = os.path.join(ROOT, "tests", "host_math", "device_math_vs_oracle.cpp")
BEGIN, END = "// ---- begin inline-PTX helpers ----", "// ---- end inline-PTX helpers ----"

# portable C++ with the definitions of the inline-PTX helpers (sign, magnitude and ordering of the
# bit patterns of doubles; the float overloads are the plain operations)
PORTABLE = r'''
static inline long long bits_(double x) { long long b; std::memcpy(&b, &x, 8); return b; }
static inline double from_bits_(long long b) { double x; std::memcpy(&x, &b, 8); return x; }
static const long long SIGN_ = (long long)0x8000000000000000ULL, MAG_ = 0x7fffffffffffffffLL;
inline double abs_b(double x) { return from_bits_(bits_(x) & MAG_); }
inline float abs_b(float x) { return std::fabs(x); }
inline double neg_b(double x) { return from_bits_(bits_(x) ^ SIGN_); }
inline float neg_b(float x) { return -x; }
inline double with_sign_b(double m, double s) { return from_bits_(bits_(m) | (bits_(s) & SIGN_)); }
inline float with_sign_b(float m, float s) { return std::copysign(m, s); }
inline double min_nn(double a, double b) { return bits_(a) < bits_(b) ? a : b; }
inline double max_nn(double a, double b) { return bits_(a) > bits_(b) ? a : b; }
inline float max_nn(float a, float b) { return a > b ? a : b; }
inline float min_nn(float a, float b) { return a < b ? a : b; }
inline bool gt_nn(double a, double b) { return bits_(a) > bits_(b); }
inline bool gt_nn(float a, float b) { return a > b; }
inline bool same_sign(double a, double b) {
  long long x = bits_(a), y = bits_(b);
  return (x ^ y) >= 0 && (x & MAG_) != 0 && (y & MAG_) != 0;
}
inline bool same_sign(float a, float b) { return a * b > 0.f; }
inline bool sign_bit_b(double x) { return bits_(x) < 0; }
inline bool sign_bit_b(float x) { return std::signbit(x); }
// approximate seeds: the correctly rounded value with its low 30 mantissa bits cleared (a relative
// error below 2^-22, like the hardware approximations'); subnormal arguments flush to zero
inline double seed_(double v) { return from_bits_(bits_(v) & ~((1LL << 30) - 1)); }
inline double ftz_(double x) { return std::fabs(x) < 2.2250738585072014e-308 ? std::copysign(0.0, x) : x; }
inline double rcp_seed(double x) { return seed_(1.0 / ftz_(x)); }
inline long long okey(double x) { long long k = bits_(x); return k ^ ((k >> 63) & MAG_); }
template <int K> inline double scale_down_b(double x) {
  const double r = x * (1.0 / (1 << K));
  return std::fabs(r) < 2.2250738585072014e-308 ? std::copysign(0.0, x) : r;
}
template <int K> inline float scale_down_b(float x) { return x * (1.0f / (float)(1 << K)); }
inline double rsqrt_seed(double x) { return seed_(1.0 / std::sqrt(ftz_(x))); }
inline unsigned umulhi32(unsigned a, unsigned b) { return (unsigned)(((unsigned long long)a * b) >> 32); }
// exp_tang's bit-pattern pieces and the FP32 operations rounded to nearest (host floats are IEEE
// single with subnormals; 1/sqrt through double, rounded once more)
inline bool exp_fast_range(double x) {
  const unsigned long long ux = (unsigned long long)bits_(x);
  return ux <= 0xc086180000000000ull && (ux >= 0x8000000000000000ull || ux < 0x4086180000000000ull);
}
inline int lo_word(double x) { return (int)(unsigned)((unsigned long long)bits_(x) & 0xffffffffull); }
inline double scale_pow2(double y, int m) { return from_bits_(bits_(y) + (long long)m * (1LL << 52)); }
inline double exp2_frac32(int j) { return kExp2Frac32[j]; }
inline float fsqrt_rn(float x) { return std::sqrt(x); }
inline float frsqrt_rn(float x) { return (float)(1.0 / std::sqrt((double)x)); }
inline float fdiv_rn(float a, float b) { return a / b; }
inline float fmul_rn(float a, float b) { return a * b; }
inline float f_inf() { return std::numeric_limits<float>::infinity(); }
'''

BOUNDS = {"ppm_lean_close": 0, "ppm_stream_bits": 0, "ppm_carried_bits": 0, "ppm_fp32": 0, "riemann_fp64": 0, "riemann_fp32": 0,
          "chemistry": 0, "heatcool": 0, "chemistry_ions": 0, "heatcool_ions": 0, "ion_instances_without_ions_same_bits": 0, "cfl": 0,
          "newton_raphson_ulp": 0, "fast_index_division": 0, "exp_tang_ulp": 0, "cfl_screen_bound": 0,
          "cfl_screen_guard_share": 0}


def _cuda_include():
    for d in [os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"]:
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    inc = _cuda_include()
    if shutil.which("g++") is None or inc is None:
        pytest.skip("needs g++ and the CUDA headers")
    from oracle import oracle as O
    lib = O.build()
    src = open(HEADER).read()
    a, b = src.index(BEGIN), src.index(END)
    tmp = tmp_path_factory.mktemp("host_math")
    copy = tmp / "mhd_device_host.cuh"
    copy.write_text(src[:a] + PORTABLE + src[b + len(END):])
    exe = tmp / "device_math_vs_oracle"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-w", f"-I{inc}",
                    f'-DMHD_DEVICE_HOST_COPY="{copy}"', HARNESS, lib, f"-Wl,-rpath,{os.path.dirname(lib)}",
                    "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=600).stdout
    res = {}
    for line in out.splitlines():
        name, n, worst, beyond = line.split()
        res[name] = (int(n), float(worst), int(beyond))
    return res


@pytest.mark.parametrize("name", sorted(BOUNDS))
def test_device_math_matches_oracle(results, name):
    n, worst, beyond = results[name]
    assert n > 0
    assert beyond == BOUNDS[name], (name, n, worst, beyond)
