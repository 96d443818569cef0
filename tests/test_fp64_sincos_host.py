"""The FP64 sin/cos helper of the generated kernels (csrc/exa_fp64_sincos.inc: Cody-Waite
reduction, minimax polynomials) compiled for the host with shims for the CUDA bit-cast intrinsics
and checked against the host C library: within 1 ulp over a sweep of arguments next to multiples
of pi/2, tiny, large and signed-zero arguments.  Host fma is correctly rounded like the device's,
so the host build computes the same values as the kernels.  The polynomial coefficients in the
helper are the ones the Remez script beside it (csrc/gen_sincos_minimax.py) derives, and that script's
error bound for them is checked independently of the script: the rounded polynomials are compared
with mpmath's sin and cos on a grid that the script does not use."""
import os
import re
import sys
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
INC = os.path.join(ROOT, "paper_2608_16265_gb300", "csrc", "exa_fp64_sincos.inc")

SHIMS = r'''
#include <cmath>
#include <cstring>
#include <cstdio>
#include <random>
#include <vector>
using std::fma; using std::fabs;
static inline long long __double_as_longlong(double d) { long long v; std::memcpy(&v, &d, 8); return v; }
static inline int __double2loint(double d) { return (int)(unsigned)(__double_as_longlong(d) & 0xffffffffLL); }
static inline int __double2hiint(double d) { return (int)(__double_as_longlong(d) >> 32); }
static inline double __hiloint2double(int hi, int lo) {
  unsigned long long v = ((unsigned long long)(unsigned)hi << 32) | (unsigned)lo; double d; std::memcpy(&d, &v, 8); return d; }
#define __device__
#define __forceinline__ inline
'''

MAIN = r'''
int main() {
  std::mt19937_64 rng(11);
  std::vector<double> v;
  for (int k = -2000; k <= 2000; k++) for (double d : {0.0, 1e-9, -1e-12, 3e-7}) v.push_back(k * (M_PI / 2) + d);
  std::uniform_real_distribution<double> u4(-4, 4), u5(-1e5, 1e5), ex(-300, 0), u6(-3e6, 3e6);
  for (int i = 0; i < 20000; i++) v.push_back(u4(rng));
  for (int i = 0; i < 20000; i++) v.push_back(u5(rng));
  for (int i = 0; i < 2000; i++) { double t = std::pow(10.0, ex(rng)); v.push_back(t); v.push_back(-t); }
  for (int i = 0; i < 200; i++) v.push_back(u6(rng));
  for (double x : {0.0, -0.0, 1048575.9, 1048576.0, 1073741824.0, 5e-324}) v.push_back(x);
  double worst = 0.0;
  for (double a : v) {
    double s, c;
    exa_sincos64(a, &s, &c);
    const double ws = std::sin(a), wc = std::cos(a);
    const double rs = ws != 0 ? std::fabs(s - ws) / std::fabs(ws) : std::fabs(s - ws);
    const double rc = std::fabs(c - wc) / std::fabs(wc);
    worst = std::fmax(worst, std::fmax(rs, rc));
  }
  double s0, c0, s1, c1;
  exa_sincos64(-0.0, &s0, &c0);
  exa_sincos64(0.0, &s1, &c1);
  std::printf("%zu %.6g %d %d %.17g %.17g\n", v.size(), worst, (int)std::signbit(s0), (int)std::signbit(s1), c0, c1);
}
'''


def test_fp64_sincos_helper_against_libm(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    text = open(INC).read()
    body = text[text.index('R"EXA(') + len('R"EXA('):text.rindex(')EXA"')]
    src = tmp_path / "t.cpp"
    src.write_text(SHIMS + body + MAIN)
    exe = tmp_path / "t"
    subprocess.run([gxx, "-O2", "-ffp-contract=off", "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    n, worst, sb0, sb1, c0, c1 = int(out[0]), float(out[1]), int(out[2]), int(out[3]), float(out[4]), float(out[5])
    assert n > 50000
    assert worst <= 2.3e-16, worst  # 1 ulp relative
    assert sb0 == 1 and sb1 == 0 and c0 == 1.0 and c1 == 1.0


def test_sincos_coefficients_are_the_remez_ones():
    mp = pytest.importorskip("mpmath")
    sys.path.insert(0, os.path.dirname(INC))
    try:
        import gen_sincos_minimax as gen
    finally:
        sys.path.pop(0)
    s_coef, c_coef = gen.derive()
    text = open(INC).read()
    lits = [float.fromhex(v) for v in re.findall(r"-?0x1\.[0-9a-f]+p[-+]?\d+", text)]
    # every derived coefficient appears in the helper, sin in S(z) and cos in C(z)
    for a in s_coef + c_coef:
        assert a in lits, a.hex()
    # independent check of the bound: relative error of the rounded polynomials against mpmath on
    # a grid offset from the script's, in 50-digit arithmetic
    mp.mp.dps = 50
    worst_s = worst_c = mp.mpf(0)
    for i in range(1, 1501):
        r = (mp.pi / 4) * (mp.mpf(i) - mp.mpf("0.37")) / 1500
        z = r * r
        ps = mp.mpf(0)
        for a in reversed(s_coef):
            ps = ps * z + mp.mpf(a)
        pc = mp.mpf(0)
        for a in reversed(c_coef):
            pc = pc * z + mp.mpf(a)
        worst_s = max(worst_s, abs((r + r * z * ps) / mp.sin(r) - 1))
        worst_c = max(worst_c, abs((1 - z / 2 + z * z * pc) / mp.cos(r) - 1))
    assert worst_s < 2.0 ** -55 and worst_c < 2.0 ** -55, (float(worst_s), float(worst_c))
