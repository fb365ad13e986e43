"""The C-ABI library loads and exports every symbol include/lqcd.h declares
(CPU only: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "lqcd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lqcd_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1701_00426_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_expected_api():
    syms = declared_symbols()
    from paper_1701_00426_gb300 import lqcd
    assert sorted(lqcd.EXPORTED) == syms


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols():
        assert hasattr(lib, name), f"{name} missing from liblqcd.so"


def test_binding_loads_and_reports_version(lib):
    from paper_1701_00426_gb300 import lqcd
    L = lqcd.load()
    assert L.lqcd_version() >= 100
    o = lqcd.default_opts()
    assert o.prec == lqcd.PREC_FP64 and o.recon == 18 and o.max_iter == 20000
    assert o.fp64_until == 3e-4 and o.check_every == 32 and o.delta_reliable == 0.1
    assert o.staged == 1 and o.pdl == 0


def test_create_rejects_odd_sides_without_gpu(lib):
    """Argument checks run before any CUDA call."""
    from paper_1701_00426_gb300 import lqcd
    L = lqcd.load()
    h = ctypes.c_void_p()
    st = L.lqcd_create((ctypes.c_int * 4)(4, 4, 3, 4), None, ctypes.byref(h))
    assert st == lqcd.LQCD_EINVAL
    assert b"even" in L.lqcd_last_error()
    o = lqcd.default_opts(recon=7)
    st = L.lqcd_create((ctypes.c_int * 4)(4, 4, 4, 4), ctypes.byref(o), ctypes.byref(h))
    assert st == lqcd.LQCD_EINVAL
    for bad in (-1e-3, 1.0):
        o = lqcd.default_opts(fp64_until=bad)
        st = L.lqcd_create((ctypes.c_int * 4)(4, 4, 4, 4), ctypes.byref(o), ctypes.byref(h))
        assert st == lqcd.LQCD_EINVAL and b"fp64_until" in L.lqcd_last_error()
    o = lqcd.default_opts(staged=2)
    st = L.lqcd_create((ctypes.c_int * 4)(4, 4, 4, 4), ctypes.byref(o), ctypes.byref(h))
    assert st == lqcd.LQCD_EINVAL and b"staged" in L.lqcd_last_error()
    o = lqcd.default_opts(pdl=-1)
    st = L.lqcd_create((ctypes.c_int * 4)(4, 4, 4, 4), ctypes.byref(o), ctypes.byref(h))
    assert st == lqcd.LQCD_EINVAL and b"pdl" in L.lqcd_last_error()


def test_no_oracle_in_product_path():
    """The product package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_1701_00426_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(from|import)\s+oracle|liboracle|lqcd_oracle|oracle_[a-z]+\(",
                                     text, flags=re.M), f


def test_fastdiv_host_matches_integer_division():
    """The magic-number division used for site decoding (compiled as host C++)."""
    import subprocess
    import tempfile
    code = r'''
#include <cstdio>
#include <cstdint>
#define __host__
#define __device__
#define __forceinline__ inline
struct float2 {float x, y;}; struct float4 {float x, y, z, w;};
''' + open(os.path.join(ROOT, "paper_1701_00426_gb300", "csrc", "common.cuh")).read().split(
        "// ------------------------------------------------------------------ df64 primitives")[0].split(
        "namespace lqcd {", 1)[1] + r'''
int main() {
  uint32_t ds[] = {1, 2, 3, 4, 5, 6, 7, 8, 10, 12, 16, 20, 24, 30, 32, 36, 48, 64, 100, 1000};
  uint64_t bad = 0;
  for (uint32_t d : ds) {
    FastDiv f = make_fastdiv(d);
    for (uint32_t n = 0; n < 3000000; n += 7) if (fdiv(n, f) != n / d) ++bad;
    for (uint32_t n = 2147483647u; n > 2147000000u; n -= 13) if (fdiv(n, f) != n / d) ++bad;
  }
  printf("%llu\n", (unsigned long long)bad);
  return bad != 0;
}
'''
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "t.cpp")
        open(src, "w").write(code)
        exe = os.path.join(td, "t")
        subprocess.run(["g++", "-std=c++17", "-O1", src, "-o", exe], check=True, capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 0 and r.stdout.strip() == "0"


def test_integer_fp64_split_host():
    """split_f64 (hi + lo floats from an IEEE double with integer operations)
    compiled as host C++: |d - hi - lo| <= 2^-48 |d| inside the exponent
    window, exact zero, and the out-of-window flag."""
    import subprocess
    import tempfile
    common = open(os.path.join(ROOT, "paper_1701_00426_gb300", "csrc", "common.cuh")).read()
    start = common.index("// Split an IEEE double into hi + lo floats")
    end = common.index("// df64 -> nearest-ish IEEE double")
    code = r'''
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <cmath>
#include <random>
#define __device__
#define __forceinline__ inline
struct float2 { float x, y; };
static inline float2 make_float2(float a, float b) { return {a, b}; }
static inline int __double2hiint(double d) { uint64_t u; memcpy(&u, &d, 8); return (int)(uint32_t)(u >> 32); }
static inline int __double2loint(double d) { uint64_t u; memcpy(&u, &d, 8); return (int)(uint32_t)u; }
static inline uint32_t __funnelshift_l(uint32_t lo, uint32_t hi, unsigned s) {
  return (uint32_t)((((uint64_t)hi << 32) | lo) << s >> 32); }
static inline float __uint_as_float(uint32_t u) { float f; memcpy(&f, &u, 4); return f; }
static inline float __fsub_rn(float a, float b) { volatile float r = a - b; return r; }
''' + common[start:end] + r'''
int main() {
  std::mt19937_64 g(7);
  long bad_err = 0, n = 0; double worst = 0;
  auto check = [&](double d) {
    bool bad = false; float2 s = split_f64(d, bad);
    if (bad) { ++bad_err; return; }
    double err = std::fabs(d - ((double)s.x + (double)s.y));
    double rel = d == 0 ? err : err / std::fabs(d);
    if (rel > worst) worst = rel;
    ++n;
  };
  std::uniform_real_distribution<double> u(-50, 50);
  for (int i = 0; i < 2000000; ++i) { double m = (g() >> 11) * 0x1p-53 + 0.5; double d = std::ldexp(m, (int)u(g)); if (g() & 1) d = -d; check(d); }
  for (int k = -55; k < 60; ++k) {              // powers of two, all-ones significands, ties
    check(std::ldexp(1.0, k)); check(-std::ldexp(1.0, k));
    check(std::nextafter(std::ldexp(1.0, k), 0.0)); check(std::nextafter(std::ldexp(1.0, k), 1e300));
    check(std::ldexp(1.0 + 0x1p-24, k)); check(std::ldexp(1.0 + 0x1p-24 + 0x1p-52, k));
    check(std::ldexp(1.0 + 3 * 0x1p-25, k)); check(std::ldexp(2.0 - 0x1p-24, k));
  }
  bool b0 = false; float2 z = split_f64(0.0, b0);
  bool b1 = false; split_f64(1e30, b1);
  bool b2 = false; split_f64(1e-30, b2);
  bool b3 = false; split_f64(-0.0, b3);
  printf("%ld %ld %.3e %d %d %d %d %g %g\n", n, bad_err, worst, (int)b0, (int)b1, (int)b2, (int)b3, z.x, z.y);
  return !(bad_err == 0 && worst <= 0x1p-48 && !b0 && b1 && b2 && !b3 && z.x == 0 && z.y == 0);
}
'''
    with tempfile.TemporaryDirectory() as td:
        src = os.path.join(td, "t.cpp")
        open(src, "w").write(code)
        exe = os.path.join(td, "t")
        subprocess.run(["g++", "-std=c++17", "-O1", "-ffp-contract=off", src, "-o", exe], check=True,
                       capture_output=True)
        r = subprocess.run([exe], capture_output=True, text=True)
        assert r.returncode == 0, r.stdout


def _entry_bodies():
    """(name, body) of every extern "C" definition under csrc/ whose first
    parameter is a context or a server."""
    csrc = os.path.join(ROOT, "paper_1701_00426_gb300", "csrc")
    out = []
    for f in sorted(os.listdir(csrc)):
        if not f.endswith(".cu"):
            continue
        src = open(os.path.join(csrc, f)).read()
        for m in re.finditer(r"^(?:extern \"C\" )?(?:int|void) (lqcd_[a-z0-9_]+)\((lqcd_ctx|lqcd_server|lqcd_ctx \*const) \*",
                             src, re.M):
            start = src.index("{", m.end())
            depth, i = 0, start
            while True:
                depth += {"{": 1, "}": -1}.get(src[i], 0)
                i += 1
                if depth == 0:
                    break
            out.append((m.group(1), src[start:i]))
    return out


# Server calls that only touch host state (queues, counters, copies of
# finished results); their device work runs on the server's own thread, which
# makes the server's device current when it starts.
HOST_ONLY_SERVER_CALLS = {"lqcd_serve_submit", "lqcd_serve_set_opts", "lqcd_serve_poll",
                          "lqcd_serve_drain", "lqcd_serve_stats_get"}


def test_every_context_call_runs_on_the_context_device():
    """Each C entry point that takes a context switches to the context's
    device for the call (and back), so a thread whose current device differs
    cannot launch on the wrong GPU."""
    bodies = _entry_bodies()
    names = {n for n, _ in bodies}
    assert {"lqcd_deo_apply", "lqcd_mscg_solve", "lqcd_deo_apply_host_noalloc",
            "lqcd_stout_force", "lqcd_rational_apply", "lqcd_serve_register_field"} <= names
    for name, body in bodies:
        if name in HOST_ONLY_SERVER_CALLS:
            continue
        assert "LQCD_ON_DEVICE(" in body or "DeviceGuard device_guard(" in body, name
