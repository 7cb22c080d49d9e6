// Specialised fused forward + adjoint kernel for one diagram.
//
// The generic fused kernel (bwd_kernel<false, true> in tami_bwd.cu) reads its term table from
// shared memory and keeps every per-sample quantity (energy combinations, Fermi values, pole-DAG
// node values, adjoints, phase-2 products) in arrays indexed by table entries, which the compiler
// must place in local memory.  Here the same computation is written out as CUDA C++ for one table:
// every table index becomes a constant and every per-sample array a set of named scalars, in the
// generic kernel's operation order (one fma per pole-DAG edge, the same phase-2 products and
// reverse sweep).  The source is compiled at run time with NVRTC for sm_103a, loaded with the
// runtime's library API and launched with the generic kernel's partial-sum layout, so the generic
// final reduction finishes it.  Values agree with the generic kernel to rounding (the compiler
// may fuse multiply-adds differently in the two codes).
//
// NVRTC is loaded with dlopen on first use; without it the generic kernel is used (or, in the
// "always" mode, the call fails with TAMI_EUNSUPPORTED).
#include <cuda_runtime.h>
#include <dlfcn.h>
#include <sys/stat.h>
#include <unistd.h>

#include <algorithm>
#include <chrono>
#include <cinttypes>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <regex>
#include <functional>
#include <atomic>
#include <memory>
#include <mutex>
#include <thread>
#include <string>
#include <vector>

#include "tami_internal.h"

#include "tami_devmath_src.inc"   // kDevmathSource: the text of tami_devmath.cuh (generated by build.py)

namespace tami {

namespace {

constexpr int kJitBlock = 128;          // threads per block of the energy-input kind (one row each)
constexpr int kJitMaxOps = 1 << 15;     // pole-DAG edges the generator writes out
constexpr int kJitMaxFreq = 256;        // frequencies (the generic adjoint's limit)

// adjoint encoding of the pole-DAG ops (see tami_internal.h)
constexpr int kDstMask = (1 << kOpbDstBits) - 1;

std::mutex g_jit_mu;
int g_jit_mode = -1;                    // TAMI_JIT_* ; -1: not yet read from $TAMI_JIT

int jit_mode() {
  std::lock_guard<std::mutex> lk(g_jit_mu);
  if (g_jit_mode < 0) {
    g_jit_mode = TAMI_JIT_AUTO;
    if (const char* e = std::getenv("TAMI_JIT")) {
      if (!std::strcmp(e, "never") || !std::strcmp(e, "0")) g_jit_mode = TAMI_JIT_NEVER;
      else if (!std::strcmp(e, "always") || !std::strcmp(e, "2")) g_jit_mode = TAMI_JIT_ALWAYS;
    }
  }
  return g_jit_mode;
}

// --------------------------------------------------------------------------- NVRTC by dlopen
struct Nvrtc {
  bool tried = false, ok = false;
  std::string why;
  typedef int (*Create)(void**, const char*, const char*, int, const char* const*, const char* const*);
  typedef int (*Compile)(void*, int, const char* const*);
  typedef int (*GetSize)(void*, size_t*);
  typedef int (*GetData)(void*, char*);
  typedef int (*Destroy)(void**);
  typedef const char* (*ErrStr)(int);
  typedef int (*Version)(int*, int*);
  std::string version;           // "nvrtc <major>.<minor>", part of every disk-cache entry's identity
  Create create = nullptr;
  Compile compile = nullptr;
  GetSize log_size = nullptr, cubin_size = nullptr;
  GetData log = nullptr, cubin = nullptr;
  Destroy destroy = nullptr;
  ErrStr err = nullptr;
};

Nvrtc& nvrtc() {
  static Nvrtc n;
  std::lock_guard<std::mutex> lk(g_jit_mu);
  if (n.tried) return n;
  n.tried = true;
  std::vector<std::string> names;
  if (const char* e = std::getenv("TAMI_NVRTC")) {
    if (!std::strcmp(e, "none")) { n.why = "NVRTC disabled ($TAMI_NVRTC=none)"; return n; }
    names.push_back(e);
  }
  names.insert(names.end(), {"libnvrtc.so.13", "/usr/local/cuda/lib64/libnvrtc.so.13", "libnvrtc.so"});
  void* h = nullptr;
  for (const std::string& s : names)
    if ((h = dlopen(s.c_str(), RTLD_NOW | RTLD_LOCAL))) break;
  if (!h) { n.why = "NVRTC (libnvrtc.so.13) not found"; return n; }
  n.create = (Nvrtc::Create)dlsym(h, "nvrtcCreateProgram");
  n.compile = (Nvrtc::Compile)dlsym(h, "nvrtcCompileProgram");
  n.log_size = (Nvrtc::GetSize)dlsym(h, "nvrtcGetProgramLogSize");
  n.log = (Nvrtc::GetData)dlsym(h, "nvrtcGetProgramLog");
  n.cubin_size = (Nvrtc::GetSize)dlsym(h, "nvrtcGetCUBINSize");
  n.cubin = (Nvrtc::GetData)dlsym(h, "nvrtcGetCUBIN");
  n.destroy = (Nvrtc::Destroy)dlsym(h, "nvrtcDestroyProgram");
  n.err = (Nvrtc::ErrStr)dlsym(h, "nvrtcGetErrorString");
  Nvrtc::Version ver = (Nvrtc::Version)dlsym(h, "nvrtcVersion");
  int major = 0, minor = 0;
  n.ok = n.create && n.compile && n.log_size && n.log && n.cubin_size && n.cubin && n.destroy && n.err && ver &&
         ver(&major, &minor) == 0;
  n.version = "nvrtc " + std::to_string(major) + "." + std::to_string(minor);
  if (!n.ok) n.why = "NVRTC lacks an expected entry point";
  return n;
}

// --------------------------------------------------------------------------- disk cache of cubins
// $TAMI_JIT_CACHE names the directory (default $HOME/.cache/libtami_jit; "none": no cache).  The
// cache is consulted only when NVRTC loads, since the compiler's version is part of every entry's
// identity.
std::string jit_cache_dir() {
  const char* p = std::getenv("TAMI_JIT_CACHE");
  if (p && !std::strcmp(p, "none")) return "";
  if (p && *p) return p;
  const char* h = std::getenv("HOME");
  return std::string(h ? h : ".") + "/.cache/libtami_jit";
}

void make_dirs(const std::string& dir) {   // mkdir -p; failures show up when the file is written
  for (size_t i = 1; i <= dir.size(); ++i)
    if (i == dir.size() || dir[i] == '/') mkdir(dir.substr(0, i).c_str(), 0755);
}

const char kCacheMagic[8] = {'T', 'A', 'M', 'I', 'J', 'I', 'T', '1'};

// --------------------------------------------------------------------------- the generator
struct Table {
  const TableHeader& h;
  const unsigned char* b;
  const int* I(int off) const { return reinterpret_cast<const int*>(b + off); }
  const double* D(int off) const { return reinterpret_cast<const double*>(b + off); }
};

std::string lit(double v) {   // exact double literal
  char buf[64];
  std::snprintf(buf, sizeof buf, "%a", v);
  return buf;
}

struct Out {
  std::string s;
  void operator()(const char* fmt, ...) __attribute__((format(printf, 2, 3))) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    std::vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    s += buf;
    s += '\n';
  }
};

// The three kinds of specialised kernel: the fused forward + adjoint (tami_forward_backward), the
// forward (tami_forward: mean and variance sums, optional per-sample values and saved rows) and the
// adjoint (tami_backward: recomputing the energies or reading the saved rows).  Each reduces into the
// per-block layout of its generic counterpart, whose final reduction kernel finishes it.
// The energy-input kind (tami_eval_energies) reads each row's base energies instead of sampling
// momenta, takes any number of external frequencies and writes every (frequency, row) value.
enum { kKindFused = kJitKindFused, kKindFwd = kJitKindFwd, kKindBwd = kJitKindBwd, kKindEnergy = kJitKindEnergy,
       kKinds = 4 };
const char* const kKernelName[kKinds] = {"tami_jit_fused", "tami_jit_fwd", "tami_jit_bwd", "tami_jit_energy"};

// Products of the frequency loop on the integer pipes (imul of tami_devmath.cuh, bit for bit the
// FP64 unit's product), unless $TAMI_JIT_INTARITH is "0".  On this GPU the FP64 unit bounds the
// specialised kernels while the integer units are mostly idle, and the two run concurrently; the
// loop's products, which feed only fmas, move there.  Measured: the order-4 bench step 59.4 ->
// 54.0 ms.  Not for large tables (over 256 pole-DAG ops), whose kernels already wait on instruction
// fetch and whose frequency loop runs few times (order 5: 1.054 -> 1.074 s, order 6: 0.80 ->
// 0.85 s with it); nor in the per-sample code, whose many live values would spill more than the
// move gains (measured 40 % slower).
// The adjoint kinds' frequency loop reads its per-sample inputs (the group weights W, the products
// p W and the frequency-free parts b of the denominators) from shared memory, [value][thread],
// through volatile loads that the compiler cannot hoist back into registers: the loop body then
// fits more of its working values in the 64 registers and spills less (order-4 fused step 53.4 ->
// 49.5 ms, order-3 real-axis workload 108.8 -> 90.9 ms; the plain forward, with fewer live values,
// gains nothing; the running sums Wbar and b-adjoint there as well measured 0.3 % slower).  $TAMI_JIT_SMEMVALS=0 keeps
// them in registers.  The slots sit in dynamic shared memory after the reduction buffer; tables
// with more than 24 such values per thread keep them in registers (24 x 8 B x 1024 threads of a
// lockstep SM = 192 KB).
int loop_value_count(const TableHeader& h) { return h.n_g2 + h.n_g2cd + h.n_cden; }
bool smem_loop_values(const TableHeader& h, bool adj, int block) {
  const char* e = std::getenv("TAMI_JIT_SMEMVALS");
  (void)block;
  return adj && !(e && !std::strcmp(e, "0")) && loop_value_count(h) <= 24;
}

// Threads per block of a specialised kernel.  The Monte Carlo kinds run in lockstep blocks: 512
// threads ($TAMI_JIT_LOCKSTEP: 256, 512 or 1024), two blocks per SM, whose warps meet at a barrier
// every $TAMI_JIT_SYNC_OPS pole-DAG steps (default 32) in the straight-line per-sample code, so
// that the warps of an SM fetch the same stretch of code at a time instead of spreading over the
// whole kernel.  A large table's kernel is far larger than the instruction caches: the order-6
// table's fused step went from 790 to 677 ms (it had waited mostly on instruction fetch); the
// order-4 step 49.7 -> 48.2 ms, order 3 on the real axis 91.1 -> 86.4 ms, order 5 1.029 ->
// 1.020 s, against 128-thread blocks without barriers.  The energy-input kind (no reduction, short
// code) keeps 128-thread blocks.
int lockstep_block(const TableHeader& h, int kind) {
  (void)h;
  if (kind == kKindEnergy) return kJitBlock;
  const char* e = std::getenv("TAMI_JIT_LOCKSTEP");
  const int b = e ? std::atoi(e) : 512;
  return (b == 256 || b == 1024) ? b : 512;
}
// Blocks per SM the kernel is compiled for: 1024 threads per SM, 64 registers each.  (128
// registers at 512 threads per SM halve the large tables' spills and change no step by more than
// 1 %: the kernels are bound by FP64 issue, not by their local-memory traffic.)  $TAMI_JIT_REGS
// (80, 128) compiles for fewer resident threads with that many registers each.
int blocks_per_sm(int block) {
  const char* e = std::getenv("TAMI_JIT_REGS");
  const int regs = e ? std::atoi(e) : 64;
  if (regs <= 64 || regs > 255) return 1024 / block;
  const int b = 65536 / (block * regs);
  return b >= 1 ? b : 1;
}
// Barrier spacing: on the order-4 table (about 120 pole-DAG steps per sample) a barrier every 32
// steps gave 47.3 ms per step, every 16 or 64 47.5-47.6 ms, and none at all (a spacing above the
// table's steps) 61.7 ms -- without a barrier per tile the warps of a block drift apart over the
// ~100 tiles each block takes and spread over the code again.
int lockstep_sync_ops() {
  const char* e = std::getenv("TAMI_JIT_SYNC_OPS");
  const int k = e ? std::atoi(e) : 32;
  return k >= 4 ? k : 32;
}

// Each group's product of real-denominator reciprocals RR is formed first and kept for the
// adjoint, W1 = pv RR, instead of W1 built factor by factor and RR formed again in the reverse
// sweep (order-6 step 676 -> 663 ms, fewer spills; order 4 unchanged).  $TAMI_JIT_KEEPRR=0 builds
// W1 factor by factor.
bool keep_rr() {
  const char* e = std::getenv("TAMI_JIT_KEEPRR");
  return !(e && !std::strcmp(e, "0"));
}

// The per-sample products of tables up to 256 pole-DAG ops (group weights, Fermi segments, the
// reverse sweep's first adjoint terms, the real denominators' adjoints) run on the integer pipes
// as well, with the call-free imul_ftz (IEEE products for normal values; subnormals flush to
// zero): order-4 step 48.07 -> 47.22 ms.  Larger tables keep them on the FP64 unit: there the
// integer product's registers double the spills (order 6: 663 -> 730 ms).  $TAMI_JIT_PSMUL=0 keeps
// every table's per-sample products on the FP64 unit, $TAMI_JIT_PSMUL=all moves them for every table,
// $TAMI_JIT_PSMUL=fwd every table's forward part (values and weights; the reverse sweep keeps the
// default).
bool ps_products(const TableHeader& h, bool reverse = false) {
  const char* e = std::getenv("TAMI_JIT_PSMUL");
  if (e && !std::strcmp(e, "all")) return true;   // every table ($TAMI_JIT_PSMUL=all)
  if (e && !std::strcmp(e, "fwd") && !reverse) return true;   // every table's forward part
  return h.n_ops <= 256 && !(e && !std::strcmp(e, "0"));
}
// The reverse sweep's sums (combination, Fermi-value and energy adjoints, each segment's sum) take
// their first term as an assignment, a copy or a product, instead of an add or fma onto 0.0 that the
// compiler must keep; $TAMI_JIT_FIRSTTERM=0 starts them from 0.0 instead.
bool first_terms() {
  const char* e = std::getenv("TAMI_JIT_FIRSTTERM");
  return !(e && !std::strcmp(e, "0"));
}
// With the per-sample products on the integer pipes, a pole-DAG chain's first step F * operand is
// one of them; $TAMI_JIT_PSFIRST=0 keeps it an fma onto 0.0 on the FP64 unit.
bool ps_first_steps() {
  const char* e = std::getenv("TAMI_JIT_PSFIRST");
  return !(e && !std::strcmp(e, "0"));
}
// a * b, on the integer pipes where the per-sample products go there
std::string pmul(bool ps, const std::string& a, const std::string& b) {
  return ps ? "imul_ftz(" + a + ", " + b + ")" : a + " * " + b;
}

// The frequency loop's products (1/D = D r, the trie's complex products, Z, the sums' first terms)
// run on the integer pipes with imul, for every table: with 32 frequencies the 85 order-2..5
// diagrams went from 2.668 to 2.255 s once the large tables (which had kept them on the FP64 unit
// while their kernels waited on instruction fetch) took them too.  $TAMI_JIT_INTARITH=0 keeps them
// on the FP64 unit.
bool int_products(const TableHeader& h) {
  (void)h;
  const char* e = std::getenv("TAMI_JIT_INTARITH");
  return !(e && !std::strcmp(e, "0"));
}

void emit_phase2(Out& o, const Table& t, int kind, bool xr_zero) {
  const TableHeader& h = t.h;
  const bool ia = int_products(h);
  const bool ps = ps_products(h) && kind != kKindEnergy;
  auto PM = [&](const std::string& a, const std::string& b) { return pmul(ps, a, b); };
  auto MUL = [&](const std::string& a, const std::string& b) {
    return ia ? "imul(" + a + ", " + b + ")" : PM(a, b);
  };
  auto NEG = [&](const std::string& a) {   // sign flip (no arithmetic)
    return "__longlong_as_double(__double_as_longlong(" + a + ") ^ (long long)0x8000000000000000ull)";
  };
  auto S = [](const char* p, int i) { return std::string(p) + std::to_string(i); };
  const bool energy = kind == kKindEnergy;
  const bool fwd = kind != kKindBwd, adj = kind == kKindFused || kind == kKindBwd;
  const int nc = h.n_cden, np = h.n_pnode;
  const int* pnode = t.I(h.off_pnode);
  const int* g2 = t.I(h.off_g2);
  const int* g2cd = t.I(h.off_g2cd);
  const int* g2node = t.I(h.off_g2node);
  const double* cden_a = t.D(h.off_cden_a);
  const int* cden_xk = t.I(h.off_cden_xk);
  o("      for (int f = 0; f < n_f; ++f) {");
  o("        const double Xr = Xs[2 * f]; (void)Xr;");
  if (adj) o("        const double gr = Gs[2 * f], gim = Gs[2 * f + 1], ngr = -gr, ngi = -gim; (void)ngr; (void)ngi;");
  for (int c = 0; c < nc; ++c) {
    if (xr_zero) o("        const double Dr%d = b%d;", c, c);
    else if (energy) o("        const double Dr%d = fma(%s, Xs[2 * (%d * n_f + f)], b%d);", c, lit(cden_a[c]).c_str(), cden_xk[c], c);
    else o("        const double Dr%d = fma(%s, Xr, b%d);", c, lit(cden_a[c]).c_str(), c);
    o("        const double r%d = rcp(fma(Dr%d, Dr%d, AXI2[%d * n_f + f]));", c, c, c, c);
    o("        const double vre%d = %s, vim%d = %s;", c, MUL(S("Dr", c), S("r", c)).c_str(), c,
      NEG(MUL("AXI[" + std::to_string(c) + " * n_f + f]", S("r", c))).c_str());
  }
  for (int k = 0; k < np; ++k) {
    const int src = pnode[2 * k], cc = pnode[2 * k + 1], v = nc + k;
    o("        const double vre%d = fma(vre%d, vre%d, %s), vim%d = fma(vre%d, vim%d, %s);", v, src, cc,
      NEG(MUL(S("vim", src), S("vim", cc))).c_str(), v, src, cc, MUL(S("vim", src), S("vre", cc)).c_str());
  }
  // sums that start at zero take their first term as a product (an addition to an exact zero is
  // no arithmetic; only the sign of a zero result can differ)
  std::vector<char> u_set(nc, 0);
  if (fwd) {
    if (h.g2_const) o("        double vr = W2_0, vi = 0.0;");
    else o("        double vr, vi;");
  }
  if (adj)
    for (int c = 0; c < nc; ++c) o("        double U_re%d = 0.0, U_im%d = 0.0;", c, c);
  bool v_set = h.g2_const != 0;
  for (int g = h.g2_const; g < h.n_g2; ++g) {
    const int v = g2node[g];
    if (fwd) {
      if (v_set) o("        vr = fma(W2_%d, vre%d, vr); vi = fma(W2_%d, vim%d, vi);", g, v, g, v);
      else o("        vr = %s; vi = %s;", MUL(S("W2_", g), S("vre", v)).c_str(), MUL(S("W2_", g), S("vim", v)).c_str());
      v_set = true;
    }
    if (adj) {
      o("        Wb2_%d = fma(gr, vre%d, fma(gim, vim%d, Wb2_%d));", g, v, v, g);
      for (int q = g2[g]; q < g2[g + 1]; ++q) {
        const int cc = g2cd[2 * q];
        if (u_set[cc])
          o("        U_re%d = fma(pW%d, vre%d, U_re%d); U_im%d = fma(pW%d, vim%d, U_im%d);", cc, q, v, cc, cc, q, v, cc);
        else
          o("        U_re%d = %s; U_im%d = %s;", cc, MUL(S("pW", q), S("vre", v)).c_str(), cc, MUL(S("pW", q), S("vim", v)).c_str());
        u_set[cc] = 1;
      }
    }
  }
  if (fwd && !v_set) o("        vr = 0.0; vi = 0.0;");
  if (adj) {
    o("        double dvr = 0.0, dvi = 0.0;");
    for (int c = 0; c < nc; ++c) {
      o("        { const double Zr = fma(vre%d, U_re%d, %s), Zi = fma(vre%d, U_im%d, %s);", c, c,
        NEG(MUL(S("vim", c), S("U_im", c))).c_str(), c, c, MUL(S("vim", c), S("U_re", c)).c_str());
      if (c == 0 && (cden_a[c] == 1.0 || cden_a[c] == -1.0))
        o("          dvr = %s; dvi = %s; bb%d = fma(ngr, Zr, fma(ngi, Zi, bb%d)); }", cden_a[c] == 1.0 ? NEG("Zr").c_str() : "Zr",
          cden_a[c] == 1.0 ? NEG("Zi").c_str() : "Zi", c, c);
      else if (c == 0)
        o("          dvr = %s; dvi = %s; bb%d = fma(ngr, Zr, fma(ngi, Zi, bb%d)); }", MUL(lit(-cden_a[c]), "Zr").c_str(),
          MUL(lit(-cden_a[c]), "Zi").c_str(), c, c);
      else
        o("          dvr = fma(%s, Zr, dvr); dvi = fma(%s, Zi, dvi); bb%d = fma(ngr, Zr, fma(ngi, Zi, bb%d)); }",
          lit(-cden_a[c]).c_str(), lit(-cden_a[c]).c_str(), c, c);
    }
    o("        if (act) {");   // a lane past the end adds and writes nothing
    o("        accX[2 * f] += dvr; accX[2 * f + 1] += dvi;");
    o("        if (ps_dX) reinterpret_cast<double2*>(ps_dX)[(size_t)f * n + s] = make_double2(dvr, dvi);");
    o("        }");
  }
  if (energy) {
    o("        reinterpret_cast<double2*>(ps_v)[(size_t)f * n + s] = make_double2(vr, vi);");
  } else if (fwd) {
    o("        if (act) {");
    o("        accV[4 * f] += vr; accV[4 * f + 1] += vi;");
    o("        accV[4 * f + 2] = fma(vr, vr, accV[4 * f + 2]); accV[4 * f + 3] = fma(vi, vi, accV[4 * f + 3]);");
    o("        if (ps_v) reinterpret_cast<double2*>(ps_v)[(size_t)f * n + s] = make_double2(vr, vi);");
    o("        }");
  }
  o("      }");
}

}  // namespace

bool jit_supported(const TableHeader& h, int kind, std::string* why) {
  if (h.n_ext != 1 && kind != kKindEnergy) { if (why) *why = "momentum sampling takes one external frequency"; return false; }
  if (h.n_ops > kJitMaxOps) { if (why) *why = "pole DAG above the generator's size limit"; return false; }
  return true;
}

// CUDA C++ source of the specialised kernel of one kind for one table.
std::string jit_source(const TableHeader& h, const unsigned char* blob, int kind) {
  // Large tables (over 256 pole-DAG ops) are written out into more code than the instruction
  // caches hold; their Fermi segments call one out-of-line copy of the exponential, reciprocal and
  // selects (smaller code; the largest order-5 table: 2.6 % faster, the order-4 table unchanged).
  const bool seg_calls = h.n_ops > 256;
  // (the energy-input kind keeps its per-row products on the FP64 unit: 1.093 -> 1.125 ms with them
  // on the integer pipes on the paper's energy-input example)
  bool ps = ps_products(h) && kind != kKindEnergy;   // the reverse sweep may set it otherwise
  auto PM = [&](const std::string& a, const std::string& b) { return pmul(ps, a, b); };
  const Table t{h, blob};
  const bool energy = kind == kKindEnergy;
  const bool fwd = kind != kKindBwd, adj = kind == kKindFused || kind == kKindBwd;
  const int* repl = t.I(h.off_repl);
  const int* lm_ptr = t.I(h.off_lm_ptr);
  const int* lm_l = t.I(h.off_lm_l);
  const double* lm_c = t.D(h.off_lm_c);
  const double* rep_aext = t.D(h.off_rep_aext);
  const int* combo_ptr = t.I(h.off_combo_ptr);
  const int* combo_j = t.I(h.off_combo_j);
  const double* combo_c = t.D(h.off_combo_c);
  const int* fseg = t.I(h.off_fseg);
  const int* fvr = t.I(h.off_fv);
  const int* rden = t.I(h.off_rden);
  const int* cden = t.I(h.off_cden);
  const double* cden_a = t.D(h.off_cden_a);
  const int* g1 = t.I(h.off_g1);
  const int* g1_tgt = t.I(h.off_g1_tgt);
  const int* opsb = t.I(h.off_opsb);
  const int* g1_node = t.I(h.off_g1_node);
  const double* leafA = t.D(h.off_leafA);
  const int* g1rd = t.I(h.off_g1rd);
  const int* g2 = t.I(h.off_g2);
  const double* g2cd_p = t.D(h.off_g2cd_p);
  const int* cden_xk = t.I(h.off_cden_xk);
  const double* xvec = t.D(h.off_xvec);
  const char* nval = kind == kKindFused ? "6 * n_f + 3" : kind == kKindBwd ? "2 * n_f + 3" : "4 * n_f";
  const int B = lockstep_block(h, kind);
  const bool ls = B != kJitBlock;
  const int sync_ops = lockstep_sync_ops();

  Out o;
  int since_sync = 0;
  auto step_sync = [&]() {   // lockstep blocks: a barrier every sync_ops pole-DAG steps
    if (ls && ++since_sync >= sync_ops) { o("    __syncthreads();"); since_sync = 0; }
  };
  o("// generated by libtami for one flattened term table, one sample per thread: %s",
    kind == kKindFused ? "forward + adjoint" : kind == kKindFwd ? "forward" : kind == kKindBwd ? "adjoint" : "energy input");
  o("#include \"tami_devmath.cuh\"");
  o("using namespace tami::dev;");
  if (h.n_cden > 0) {
    std::string a, k;
    for (int c = 0; c < h.n_cden; ++c) {
      a += (c ? ", " : "") + lit(cden_a[c]);
      k += (c ? ", " : "") + std::to_string(cden_xk[c]);
    }
    o("__device__ const double kJitCdenA[%d] = {%s};", h.n_cden, a.c_str());
    o("__device__ const int kJitCdenXk[%d] = {%s};", h.n_cden, k.c_str());
  }
  if (energy && h.n_ext > 1) {
    std::string v;
    for (int i = 0; i < h.n_xk * h.n_ext; ++i) v += (i ? ", " : "") + lit(xvec[i]);
    o("__device__ const double kJitXvec[%d] = {%s};", h.n_xk * h.n_ext, v.c_str());
  }
  if (seg_calls) {
    // one out-of-line copy of a Fermi segment's exponential, reciprocal and selects (smaller code)
    for (int bose = 0; bose < 2; ++bose) {
      o("static __device__ __noinline__ double2 tami_seg_%s(double xv, double beta) {", bose ? "bose" : "fermi");
      o("  double em = 0.0;");
      o("  const double y = exp_neg<%s>(%s, em); (void)em;", bose ? "true" : "false", PM("-beta", "fabs(xv)").c_str());
      o("  const double rD = rcp(%s);", bose ? "-em" : "1.0 + y");
      o("  const double t2 = %s;", PM(bose ? "(-y)" : "(y)", "rD").c_str());
      o("  const bool neg = __double_as_longlong(xv) <= 0;");
      o("  return make_double2(neg ? rD : t2, neg ? t2 : rD);");
      o("}");
    }
  }
  o("extern \"C\" __global__ void __launch_bounds__(%d, %d) %s(double lt, double ltp, double lmu, double lkx, double lky,",
    B, kind == kKindEnergy ? 8 : blocks_per_sm(B), kKernelName[kind]);
  o("    unsigned long long seed, unsigned long long offset, long long n, const double* X, const double* G, int n_f,");
  o("    double beta, double* ps_dX, double* ps_grad, double* ps_v, double* saved, double* partial, const double* P) {");
  o("  extern __shared__ __align__(16) double smem[];");
  o("  const int tid = threadIdx.x;");
  // a launch captured once in a graph reads (t, t', mu, kx, ky, beta) from device memory
  o("  if (P) { lt = P[0]; ltp = P[1]; lmu = P[2]; lkx = P[3]; lky = P[4]; beta = P[5]; }");
  if (energy) {
    // Xs [n_xk][n_f][2]: the frequencies as the denominators see them, Y_kf = sum_q v_kq X_fq
    o("  double* Xs = smem; double* AXI = Xs + %d * n_f; double* AXI2 = AXI + %d * n_f;", 2 * h.n_xk, h.n_cden);
    o("  (void)AXI; (void)AXI2; (void)G; (void)ps_dX; (void)ps_grad; (void)partial; (void)seed; (void)offset;");
    o("  (void)lt; (void)ltp; (void)lmu; (void)lkx; (void)lky;");
    if (h.n_ext == 1) {
      o("  for (int i = tid; i < 2 * n_f; i += %d) Xs[i] = X[i];", B);
    } else {
      o("  for (int i = tid; i < %d * n_f; i += %d) {", h.n_xk, B);
      o("    const int k = i / n_f, f = i %% n_f;");
      o("    const double* v = kJitXvec + k * %d; const double* x = X + 2 * (size_t)f * %d;", h.n_ext, h.n_ext);
      o("    double re = v[0] * x[0], im = v[0] * x[1];");
      o("    for (int q = 1; q < %d; ++q) { re = fma(v[q], x[2 * q], re); im = fma(v[q], x[2 * q + 1], im); }", h.n_ext);
      o("    Xs[2 * i] = re; Xs[2 * i + 1] = im;");
      o("  }");
    }
  } else {
    o("  double* Xs = smem; double* Gs = Xs + 2 * n_f; double* AXI = Gs + 2 * n_f; double* AXI2 = AXI + %d * n_f;", h.n_cden);
    o("  double* red = AXI2 + %d * n_f;", h.n_cden);
    if (smem_loop_values(h, adj, B)) o("  volatile double* jsv = red + %d;", B);   // after the [warp][32] buffer
    o("  (void)AXI; (void)AXI2; (void)G; (void)ps_dX; (void)ps_grad; (void)ps_v; (void)saved;");
    o("  for (int i = tid; i < 2 * n_f; i += %d) { Xs[i] = X[i]; Gs[i] = %s; }", B, adj ? "G[i]" : "0.0");
  }
  if (adj) {
    o("  double accX[%d];", 2 * kJitMaxFreq);
    o("  for (int i = 0; i < 2 * n_f; ++i) accX[i] = 0.0;");
    o("  double gmu = 0.0, gkx = 0.0, gky = 0.0;");
    o("  __shared__ double s_gsum;");
  }
  if (fwd && !energy) {
    o("  double accV[%d];", 4 * kJitMaxFreq);
    o("  for (int i = 0; i < 4 * n_f; ++i) accV[i] = 0.0;");
  }
  o("  __syncthreads();");
  o("  bool xr_zero;");
  o("  {");
  o("    int nonzero = 0;");
  if (h.n_cden > 0) {
    o("    for (int i = tid; i < %d * n_f; i += %d) {", h.n_cden, B);
    if (energy) o("      const double a = kJitCdenA[i / n_f] * Xs[2 * (kJitCdenXk[i / n_f] * n_f + i %% n_f) + 1];");
    else o("      const double a = kJitCdenA[i / n_f] * Xs[2 * (i %% n_f) + 1];");
    o("      AXI[i] = a; AXI2[i] = a * a;");
    o("    }");
  }
  o("    for (int i = tid; i < %d * n_f; i += %d) nonzero |= Xs[2 * i] != 0.0;", energy ? h.n_xk : 1, B);
  if (adj) o("    if (tid == 0) { double g = 0.0; for (int f = 0; f < n_f; ++f) g += Gs[2 * f]; s_gsum = g; }");
  o("    xr_zero = !__syncthreads_or(nonzero);");
  o("  }");
  o("  const long long n_tiles = (n + %d) / %d;", B - 1, B);
  o("  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {");
  if (ls) {
    // every thread reaches every barrier: a lane past the end runs the last sample again and
    // neither adds nor writes
    o("    const long long s0 = tile * %d + tid;", B);
    o("    const bool act = s0 < n;");
    o("    const long long s = act ? s0 : n - 1;");
  } else {
    o("    const long long s = tile * %d + tid;", B);
    o("    if (s >= n) continue;");
  }
  // ---- line energies: from the momenta, or (adjoint) from the forward's saved rows
  for (int r = 0; r < h.n_rep; ++r) o("    double E%d;", repl[r]);
  if (adj) for (int r = 0; r < h.n_rep_ext; ++r) o("    double Gx%d, Gy%d;", r, r);
  if (energy) {
    o("    {");
    for (int r = 0; r < h.n_rep; ++r) o("      E%d = saved[(size_t)s * %d + %d];", repl[r], h.N, repl[r]);
  } else if (kind == kKindBwd) {
    o("    if (saved) {");
    for (int r = 0; r < h.n_rep; ++r) o("      E%d = saved[(size_t)%d * n + s];", repl[r], r);
    for (int r = 0; r < h.n_rep_ext; ++r)
      o("      Gx%d = saved[(size_t)%d * n + s]; Gy%d = saved[(size_t)%d * n + s];", r, h.n_rep + 2 * r, r,
        h.n_rep + 2 * r + 1);
    o("    } else {");
  } else {
    o("    {");
  }
  if (!energy) {
  o("    const unsigned long long sg = offset + (unsigned long long)s;");
  for (int l = 0; l < h.m; ++l) {
    o("    double kx%d, ky%d;", l, l);
    o("    { unsigned int c[4] = {(unsigned int)sg, (unsigned int)(sg >> 32), %du, 0u};", l);
    o("      philox4x32_10(c, (unsigned int)seed, (unsigned int)(seed >> 32));");
    o("      kx%d = to_momentum(c[0], c[1]); ky%d = to_momentum(c[2], c[3]); }", l, l);
  }
  o("    const double kx%d = lkx, ky%d = lky; (void)kx%d; (void)ky%d;", h.m, h.m, h.m, h.m);
  for (int r = 0; r < h.n_rep; ++r) {
    const int j = repl[r];
    // a sum that starts with a +-1 label starts as that momentum (no addition to an exact zero)
    int q0 = lm_ptr[r];
    if (q0 < lm_ptr[r + 1] && (lm_c[q0] == 1.0 || lm_c[q0] == -1.0)) {
      const char* sg = lm_c[q0] > 0 ? "" : "-";
      o("    double ax%d = %skx%d, ay%d = %sky%d;", r, sg, lm_l[q0], r, sg, lm_l[q0]);
      ++q0;
    } else {
      o("    double ax%d = 0.0, ay%d = 0.0;", r, r);
    }
    for (int q = q0; q < lm_ptr[r + 1]; ++q)
      o("    ax%d = fma(%s, kx%d, ax%d); ay%d = fma(%s, ky%d, ay%d);", r, lit(lm_c[q]).c_str(), lm_l[q], r, r,
        lit(lm_c[q]).c_str(), lm_l[q], r);
    if (r < h.n_rep_ext && adj) {
      o("    E%d = line_energy_grad(ax%d, ay%d, lt, ltp, lmu, Gx%d, Gy%d);", j, r, r, r, r);
    } else if (r < h.n_rep_ext) {   // forward: the dE/dK factors only when the rows are saved (same E bits)
      o("    if (saved) { double gx, gy; E%d = line_energy_grad(ax%d, ay%d, lt, ltp, lmu, gx, gy);", j, r, r);
      o("      if (act) { saved[(size_t)%d * n + s] = gx; saved[(size_t)%d * n + s] = gy; } }", h.n_rep + 2 * r,
        h.n_rep + 2 * r + 1);
      o("    else E%d = line_energy(ax%d, ay%d, lt, ltp, lmu);", j, r, r);
    } else {
      o("    E%d = line_energy(ax%d, ay%d, lt, ltp, lmu);", j, r, r);
    }
  }
  if (kind == kKindFwd) {
    o("    if (saved && act) {");
    for (int r = 0; r < h.n_rep; ++r) o("      saved[(size_t)%d * n + s] = E%d;", r, repl[r]);
    o("    }");
  }
  }  // !energy
  o("    }");
  // ---- energy combinations
  for (int u = 0; u < h.n_combo; ++u) {
    int q0 = combo_ptr[u];
    if (q0 < combo_ptr[u + 1] && (combo_c[q0] == 1.0 || combo_c[q0] == -1.0)) {
      o("    double x%d = %sE%d;", u, combo_c[q0] > 0 ? "" : "-", combo_j[q0]);
      ++q0;
    } else {
      o("    double x%d = 0.0;", u);
    }
    for (int q = q0; q < combo_ptr[u + 1]; ++q)
      o("    x%d = fma(%s, E%d, x%d);", u, lit(combo_c[q]).c_str(), combo_j[q], u);
  }
  // ---- Fermi/Bose values (and, for the adjoint, their next derivatives), segment by segment
  for (int b = 0; b < h.n_fseg; ++b) {
    const int* sgm = fseg + 8 * b;
    const bool bose = b < h.n_fseg_bose;
    // d1 = -beta g h: the k = 0 values' derivatives (adjoint) and every k = 1 value of the segment
    // (g and h alike: the first derivative is symmetric in them)
    bool has_k1 = false;
    for (int v = sgm[3]; v < sgm[4]; ++v) has_k1 |= fvr[2 * v + 1] == 1;
    const std::string d1 = (adj || has_k1)
        ? PM("-beta", ps ? PM("sg" + std::to_string(b) + "_g", "sg" + std::to_string(b) + "_h")
                         : "(sg" + std::to_string(b) + "_g * sg" + std::to_string(b) + "_h)")
        : std::string("0.0");
    o("    double sg%d_g, sg%d_h, sg%d_d1;", b, b, b);
    if (seg_calls) {
      o("    { const double2 gh = tami_seg_%s(x%d, beta);", bose ? "bose" : "fermi", sgm[0]);
      o("      sg%d_g = gh.x; sg%d_h = gh.y; sg%d_d1 = %s; }", b, b, b, d1.c_str());
    } else {
    o("    { const double xv = x%d; double em = 0.0;", sgm[0]);
    o("      const double y = exp_neg<%s>(%s, em); (void)em;", bose ? "true" : "false", PM("-beta", "fabs(xv)").c_str());
    o("      const double rD = rcp(%s);", bose ? "-em" : "1.0 + y");
    o("      const double t2 = %s;", PM(bose ? "(-y)" : "(y)", "rD").c_str());
    o("      const bool neg = __double_as_longlong(xv) <= 0;");
    o("      sg%d_g = neg ? rD : t2; sg%d_h = neg ? t2 : rD; sg%d_d1 = %s; }", b, b, b, d1.c_str());
    }
    for (int v = sgm[2]; v < sgm[3]; ++v) {
      o("    const double fv%d = sg%d_%c;", v, b, fvr[2 * v] > 0 ? 'g' : 'h');
      if (adj) o("    const double fvd%d = sg%d_d1;", v, b);
    }
    // the adjoint's second derivative d2 = -beta d1 (h - g) = beta^2 g h (h - g), once per segment
    // with k = 1 values (an h value's is -d2)
    if (adj && has_k1)
      o("    const double sg%d_d2 = %s;", b,
        PM(PM("-beta", "sg" + std::to_string(b) + "_d1"), "(sg" + std::to_string(b) + "_h - sg" + std::to_string(b) + "_g)").c_str());
    for (int v = sgm[3]; v < sgm[4]; ++v) {
      const bool pos = fvr[2 * v] > 0;
      const int k = fvr[2 * v + 1];
      const char g = pos ? 'g' : 'h', hh = pos ? 'h' : 'g';
      if (k == 1) o("    const double fv%d = sg%d_d1;", v, b);
      else o("    const double fv%d = fermi_poly(%d, sg%d_%c, sg%d_%c, beta);", v, k, b, g, b, hh);
      if (adj && k == 1) o("    const double fvd%d = %ssg%d_d2;", v, pos ? "" : "-", b);
      else if (adj) o("    const double fvd%d = fermi_poly(%d, sg%d_%c, sg%d_%c, beta);", v, k + 1, b, g, b, hh);
    }
  }
  for (int i = 0; i < h.n_rden; ++i) o("    const double rr%d = rcp(x%d);", i, rden[2 * i]);
  // ---- pole DAG: one variable per distinct prefix of the nodes' fma chains (shared partial sums
  // once, a chain and its sign-flipped twin one variable, the twin read through a free operand
  // negation; operands that are identically zero left out, and with them the groups whose terms all
  // cancelled), group weights
  // Sums take their first term as an assignment (a copy or a product) instead of an add onto 0.0,
  // which the compiler must keep (0.0 + x is not x for x = -0.0): W2 here, and the reverse sweep's
  // adjoints below.  A sum that receives nothing is set to 0.0 where it is read.
  for (int g = 0; g < h.n_g2; ++g) o("    double W2_%d;", g);
  std::vector<char> has_w2(h.n_g2, 0);
  const DagPrefixes dp = dag_prefixes(opsb, h.n_ops, leafA);
  // a group root's value: its prefix with the root's sign
  auto root_pv = [&](int gi) {
    const int nd = g1_node[gi];
    return std::string(dp.node_sign[nd] < 0 ? "-pv" : "pv") + std::to_string(dp.node_value[nd]);
  };
  for (int gi = 0; gi < h.n_g1; ++gi) {
    for (int op = g1[4 * gi]; op < g1[4 * gi + 1]; ++op) {
      if (!dp.op_new[op]) continue;
      const int k = dp.op_prefix[op];
      const DagPrefix& q = dp.p[k];
      const double c = q.node ? 0.0 : q.osign * leafA[q.operand];
      const std::string opnd = q.node ? (q.osign < 0 ? "-pv" : "pv") + std::to_string(q.operand) : lit(c);
      const std::string add = q.parent < 0 ? "0.0" : "pv" + std::to_string(q.parent);
      if (q.parent < 0 && !q.node && (c == 1.0 || c == -1.0))
        o("    const double pv%d = %sfv%d;", k, c > 0 ? "" : "-", q.fv);   // +-F, no arithmetic
      else if (q.parent < 0 && ps && ps_first_steps())   // a chain's first step is a product
        o("    const double pv%d = %s;", k, PM("fv" + std::to_string(q.fv), opnd).c_str());
      else
        o("    const double pv%d = fma(fv%d, %s, %s);", k, q.fv, opnd.c_str(), add.c_str());
      step_sync();
    }
    if (dp.node_value[g1_node[gi]] < 0) continue;   // every term of the group cancelled: weight 0
    if (keep_rr() && g1[4 * gi + 2] < g1[4 * gi + 3]) {
      bool first = true;
      for (int q = g1[4 * gi + 2]; q < g1[4 * gi + 3]; ++q)
        for (int pw = g1rd[2 * q + 1]; pw > 0; --pw) {
          if (first) o("    double RR_%d = rr%d;", gi, g1rd[2 * q]);
          else if (ps) o("    RR_%d = imul_ftz(RR_%d, rr%d);", gi, gi, g1rd[2 * q]);
          else o("    RR_%d *= rr%d;", gi, g1rd[2 * q]);
          first = false;
        }
      o("    double W1_%d = %s;", gi, PM(root_pv(gi), "RR_" + std::to_string(gi)).c_str());
    } else {
      o("    double W1_%d = %s;", gi, root_pv(gi).c_str());
      for (int q = g1[4 * gi + 2]; q < g1[4 * gi + 3]; ++q)
        for (int pw = g1rd[2 * q + 1]; pw > 0; --pw) {
          if (ps) o("    W1_%d = imul_ftz(W1_%d, rr%d);", gi, gi, g1rd[2 * q]);
          else o("    W1_%d *= rr%d;", gi, g1rd[2 * q]);
        }
    }
    o(has_w2[g1_tgt[gi]] ? "    W2_%d += W1_%d;" : "    W2_%d = W1_%d;", g1_tgt[gi], gi);
    has_w2[g1_tgt[gi]] = 1;
  }
  for (int g = 0; g < h.n_g2; ++g)
    if (!has_w2[g]) o("    W2_%d = 0.0;", g);
  for (int c = 0; c < h.n_cden; ++c) o("    const double b%d = %sx%d;", c, cden[2 * c + 1] > 0 ? "" : "-", cden[2 * c]);
  if (adj) {
    for (int g = 0; g < h.n_g2; ++g) {
      o("    double Wb2_%d = 0.0;", g);
      for (int q = g2[g]; q < g2[g + 1]; ++q) {
        if (ps && (g2cd_p[q] == 1.0 || g2cd_p[q] == -1.0))
          o("    const double pW%d = %sW2_%d;", q, g2cd_p[q] > 0 ? "" : "-", g);
        else
          o("    const double pW%d = %s;", q, PM(lit(g2cd_p[q]), "W2_" + std::to_string(g)).c_str());
      }
    }
    for (int c = 0; c < h.n_cden; ++c) o("    double bb%d = 0.0;", c);
  }
  // ---- phase 2 over frequencies (the adjoint kinds' loop inputs in shared memory, see
  // smem_loop_values)
  const bool sv = smem_loop_values(h, adj, B);
  const int n_sv = h.n_g2 + h.n_g2cd + h.n_cden;
  if (sv) {
    for (int g = 0; g < h.n_g2; ++g) o("    jsv[%d * %d + tid] = W2_%d;", g, B, g);
    for (int q = 0; q < h.n_g2cd; ++q) o("    jsv[%d * %d + tid] = pW%d;", h.n_g2 + q, B, q);
    for (int c = 0; c < h.n_cden; ++c) o("    jsv[%d * %d + tid] = b%d;", n_sv - h.n_cden + c, B, c);
  }
  const size_t loop0 = o.s.size();
  o("    if (xr_zero) {");
  emit_phase2(o, t, kind, true);
  o("    } else {");
  emit_phase2(o, t, kind, false);
  o("    }");
  if (sv) {
    std::string loop = o.s.substr(loop0);
    auto rename = [&](const char* pat, int base) {
      const std::regex re(pat);
      std::string out;
      std::sregex_iterator it(loop.begin(), loop.end(), re), end;
      size_t last = 0;
      for (; it != end; ++it) {
        out += loop.substr(last, it->position() - last);
        out += "jsv[" + std::to_string(base + std::stoi((*it)[1].str())) + " * " + std::to_string(B) + " + tid]";
        last = it->position() + it->length();
      }
      out += loop.substr(last);
      loop.swap(out);
    };
    rename("\\bW2_(\\d+)\\b", 0);
    rename("\\bpW(\\d+)\\b", h.n_g2);
    rename("\\bb(\\d+)\\b", n_sv - h.n_cden);
    o.s.resize(loop0);
    o.s += loop;
  }
  if (adj) {
    if (h.g2_const) o("    Wb2_0 = s_gsum;");
    // ---- reverse sweep
    ps = ps_products(h, true) && kind != kKindEnergy;
    const bool ft = first_terms();
    for (int u = 0; u < h.n_combo; ++u) o(ft ? "    double xbar%d;" : "    double xbar%d = 0.0;", u);
    for (int v = 0; v < h.n_fv; ++v) o(ft ? "    double fvbar%d;" : "    double fvbar%d = 0.0;", v);
    std::vector<char> hx(h.n_combo, ft ? 0 : 1), hf(h.n_fv, ft ? 0 : 1);   // the adjoint has its first term
    for (int c = 0; c < h.n_cden; ++c) {
      const int u = cden[2 * c];
      o(hx[u] ? "    xbar%d += %sbb%d;" : "    xbar%d = %sbb%d;", u, cden[2 * c + 1] > 0 ? "" : "-", c);
      hx[u] = 1;
    }
    // pole DAG backwards: the group roots seeded with their weights' adjoints, then the prefixes in
    // reverse creation order (every contribution to a prefix's adjoint comes from a later prefix)
    std::vector<char> has(dp.p.size(), 0);
    for (int gi = h.n_g1 - 1; gi >= 0; --gi) {
      const int rp = dp.node_value[g1_node[gi]];
      if (rp < 0) continue;   // a zero weight: no adjoint to pass on
      if (!has[rp]) o("    double bp%d;", rp);
      o("    {");
      const bool kept = keep_rr() && g1[4 * gi + 2] < g1[4 * gi + 3];
      // wb: the adjoint of the root's value; the root's prefix gets it with the root's sign
      const char* rs = dp.node_sign[g1_node[gi]] < 0 ? "-" : "";
      if (kept) o("      const double wb = Wb2_%d; const double RR = RR_%d;", g1_tgt[gi], gi);
      else o("      const double wb = Wb2_%d; double RR = 1.0;", g1_tgt[gi]);
      for (int q = g1[4 * gi + 2]; q < g1[4 * gi + 3]; ++q) {
        const int i = g1rd[2 * q], pw = g1rd[2 * q + 1];
        if (!kept) for (int k = 0; k < pw; ++k) o("      RR *= rr%d;", i);
        const int u = rden[2 * i];
        if (ps) {   // wb W1 once per group, then one fma per factor
          if (q == g1[4 * gi + 2]) o("      const double tw = %s;", PM("wb", "W1_" + std::to_string(gi)).c_str());
          const std::string tp = pw == 1 ? "tw" : PM("tw", lit((double)pw));
          if (hx[u]) o("      xbar%d = fma(-%s, rr%d, xbar%d);", u, tp.c_str(), i, u);
          else o("      xbar%d = %s;", u, PM("-" + tp, "rr" + std::to_string(i)).c_str());
        } else {
          if (hx[u]) o("      xbar%d -= wb * W1_%d * %s * rr%d;", u, gi, lit((double)pw).c_str(), i);
          else o("      xbar%d = -(wb * W1_%d * %s * rr%d);", u, gi, lit((double)pw).c_str(), i);
        }
        hx[u] = 1;
      }
      if (has[rp]) o("      bp%d = fma(%swb, RR, bp%d);", rp, rs, rp);
      else o("      bp%d = %s;", rp, PM(std::string(rs) + "wb", "RR").c_str());
      has[rp] = 1;
      o("    }");
    }
    for (int k = (int)dp.p.size() - 1; k >= 0; --k) {
      if (!has[k]) continue;
      step_sync();
      const DagPrefix& q = dp.p[k];
      if (q.node) {   // the operand enters with its sign osign: so do both of its adjoint terms
        const char* os = q.osign < 0 ? "-" : "";
        if (hf[q.fv]) o("    fvbar%d = fma(%spv%d, bp%d, fvbar%d);", q.fv, os, q.operand, k, q.fv);
        else o("    fvbar%d = %s;", q.fv, PM(os + ("pv" + std::to_string(q.operand)), "bp" + std::to_string(k)).c_str());
        hf[q.fv] = 1;
        if (has[q.operand]) o("    bp%d = fma(%sfv%d, bp%d, bp%d);", q.operand, os, q.fv, k, q.operand);
        else o("    double bp%d = %s;", q.operand, PM(os + ("fv" + std::to_string(q.fv)), "bp" + std::to_string(k)).c_str());
        has[q.operand] = 1;
      } else {
        const double c = q.osign * leafA[q.operand];
        if (hf[q.fv]) o("    fvbar%d = fma(%s, bp%d, fvbar%d);", q.fv, lit(c).c_str(), k, q.fv);
        else if (c == 1.0 || c == -1.0) o("    fvbar%d = %sbp%d;", q.fv, c > 0 ? "" : "-", k);
        else o("    fvbar%d = %s;", q.fv, PM(lit(c), "bp" + std::to_string(k)).c_str());
        hf[q.fv] = 1;
      }
      if (q.parent >= 0) {
        if (has[q.parent]) o("    bp%d += bp%d;", q.parent, k);
        else o("    double bp%d = bp%d;", q.parent, k);
        has[q.parent] = 1;
      }
    }
    // each segment's Fermi values pass their adjoints to the combination: x-adjoint += sum over
    // the values of +-fvbar P_{k+1} (the sign: h = 1 - g enters with -1)
    for (int b = 0; b < h.n_fseg; ++b) {
      const int* sgm = fseg + 8 * b;
      bool any = false;
      for (int v = sgm[2]; v < sgm[4]; ++v) any |= hf[v] != 0;
      if (!any) continue;
      o("    {");
      bool first = ft;
      if (!ft) o("      double acc = 0.0;");
      for (int v = sgm[2]; v < sgm[4]; ++v) {
        if (!hf[v]) continue;
        const char* sg = fvr[2 * v] > 0 ? "" : "-";
        if (first) o("      double acc = %s;", PM(sg + ("fvbar" + std::to_string(v)), "fvd" + std::to_string(v)).c_str());
        else o("      acc = fma(%sfvbar%d, fvd%d, acc);", sg, v, v);
        first = false;
      }
      o(hx[sgm[0]] ? "      xbar%d += acc;" : "      xbar%d = acc;", sgm[0]);
      hx[sgm[0]] = 1;
      o("    }");
    }
    std::vector<char> hE(h.N, ft ? 0 : 1);
    for (int r = 0; r < h.n_rep; ++r) o(ft ? "    double Ebar%d;" : "    double Ebar%d = 0.0;", repl[r]);
    for (int u = 0; u < h.n_combo; ++u) {
      if (!hx[u]) continue;   // no adjoint reached this combination
      for (int q = combo_ptr[u]; q < combo_ptr[u + 1]; ++q) {
        const int j = combo_j[q];
        const double c = combo_c[q];
        if (hE[j]) o("    Ebar%d = fma(xbar%d, %s, Ebar%d);", j, u, lit(c).c_str(), j);
        else if (c == 1.0 || c == -1.0) o("    Ebar%d = %sxbar%d;", j, c > 0 ? "" : "-", u);
        else o("    Ebar%d = %s;", j, PM("xbar" + std::to_string(u), lit(c)).c_str());
        hE[j] = 1;
      }
    }
    for (int r = 0; r < h.n_rep; ++r)
      if (!hE[repl[r]]) o("    Ebar%d = 0.0;", repl[r]);
    o("    double mub = Ebar%d, kxb = 0.0, kyb = 0.0;", repl[0]);
    for (int r = 1; r < h.n_rep; ++r) o("    mub += Ebar%d;", repl[r]);
    for (int r = 0; r < h.n_rep_ext; ++r)
      if (r) o("    { const double eb = Ebar%d, ae = %s; kxb = fma(-eb * ae, Gx%d, kxb); kyb = fma(-eb * ae, Gy%d, kyb); }",
               repl[r], lit(rep_aext[r]).c_str(), r, r);
      else o("    { const double eb = Ebar%d, ae = %s; kxb = %s; kyb = %s; }", repl[r], lit(rep_aext[r]).c_str(),
             PM("(-eb * ae)", "Gx" + std::to_string(r)).c_str(), PM("(-eb * ae)", "Gy" + std::to_string(r)).c_str());
    o("    if (act) {");
    o("      gmu += mub; gkx += kxb; gky += kyb;");
    o("      if (ps_grad) { ps_grad[3 * s] = mub; ps_grad[3 * s + 1] = kxb; ps_grad[3 * s + 2] = kyb; }");
    o("    }");
  }
  o("  }");
  if (energy) {   // every value is an output; nothing is reduced
    o("}");
    return o.s;
  }
  // ---- block reduction into the generic kernel's per-block layout
  o("  const int nval = %s, warp = tid >> 5, lane = tid & 31;", nval);
  o("  for (int i = 0; i < nval; ++i) {");
  if (kind == kKindFused) {
    o("    double v = i < 2 * n_f ? accX[i] : (i == 2 * n_f ? gmu : (i == 2 * n_f + 1 ? gkx : gky));");
    o("    if (i >= 2 * n_f + 3) v = accV[i - 2 * n_f - 3];");
  } else if (kind == kKindBwd) {
    o("    const double v0 = i < 2 * n_f ? accX[i] : (i == 2 * n_f ? gmu : (i == 2 * n_f + 1 ? gkx : gky));");
    o("    double v = v0;");
  } else {
    o("    double v = accV[i];");
  }
  o("    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);");
  // 32 values at a time through a [warp][32] buffer
  o("    if (lane == 0) red[warp * 32 + (i & 31)] = v;");
  o("    if ((i & 31) == 31 || i == nval - 1) {");
  o("      __syncthreads();");
  o("      if (tid <= (i & 31)) {");
  o("        double u = 0.0;");
  o("        for (int w = 0; w < %d; ++w) u += red[w * 32 + tid];", B / 32);
  o("        partial[(size_t)blockIdx.x * nval + (i & ~31) + tid] = u;");
  o("      }");
  o("      __syncthreads();");
  o("    }");
  o("  }");
  o("}");
  return o.s;
}

// --------------------------------------------------------------------------- disk cache entries
uint64_t jit_fnv1a(const void* p, size_t n, uint64_t h) {
  const unsigned char* c = static_cast<const unsigned char*>(p);
  for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
  return h;
}

// Entry layout: magic (8 bytes), identity length (u64), identity, cubin length (u64), cubin,
// FNV-1a 64 of identity then cubin (u64).
bool jit_cache_read(const std::string& path, const std::string& ident, std::vector<char>* cubin) {
  FILE* f = std::fopen(path.c_str(), "rb");
  if (!f) return false;
  std::vector<char> buf;
  char chunk[65536];
  size_t got;
  while ((got = std::fread(chunk, 1, sizeof chunk, f)) > 0 && buf.size() <= (size_t(64) << 20))
    buf.insert(buf.end(), chunk, chunk + got);
  std::fclose(f);
  size_t at = 0;
  auto take_u64 = [&](uint64_t* v) {
    if (buf.size() - at < 8) return false;
    std::memcpy(v, buf.data() + at, 8);
    at += 8;
    return true;
  };
  uint64_t n_ident = 0, n_cubin = 0, sum = 0;
  if (buf.size() < 8 || std::memcmp(buf.data(), kCacheMagic, 8)) return false;
  at = 8;
  if (!take_u64(&n_ident) || n_ident != ident.size() || buf.size() - at < n_ident) return false;
  if (std::memcmp(buf.data() + at, ident.data(), n_ident)) return false;
  at += n_ident;
  if (!take_u64(&n_cubin) || n_cubin == 0 || buf.size() - at < n_cubin) return false;
  const char* cb = buf.data() + at;
  at += n_cubin;
  if (!take_u64(&sum) || at != buf.size()) return false;
  if (sum != jit_fnv1a(cb, n_cubin, jit_fnv1a(ident.data(), ident.size()))) return false;
  cubin->assign(cb, cb + n_cubin);
  return true;
}

bool jit_cache_write(const std::string& path, const std::string& ident, const std::vector<char>& cubin) {
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos && slash > 0) make_dirs(path.substr(0, slash));
  const std::string tmp = path + ".tmp" + std::to_string((long long)getpid()) + "_" +
                          std::to_string(std::hash<std::thread::id>{}(std::this_thread::get_id()));
  FILE* f = std::fopen(tmp.c_str(), "wb");
  if (!f) return false;
  const uint64_t n_ident = ident.size(), n_cubin = cubin.size();
  const uint64_t sum = jit_fnv1a(cubin.data(), cubin.size(), jit_fnv1a(ident.data(), ident.size()));
  bool ok = std::fwrite(kCacheMagic, 1, 8, f) == 8 && std::fwrite(&n_ident, 8, 1, f) == 1 &&
            std::fwrite(ident.data(), 1, ident.size(), f) == ident.size() && std::fwrite(&n_cubin, 8, 1, f) == 1 &&
            std::fwrite(cubin.data(), 1, cubin.size(), f) == cubin.size() && std::fwrite(&sum, 8, 1, f) == 1;
  ok = (std::fclose(f) == 0) && ok;
  if (ok) ok = std::rename(tmp.c_str(), path.c_str()) == 0;
  if (!ok) std::remove(tmp.c_str());
  return ok;
}

// --------------------------------------------------------------------------- compile, cache, launch
struct JitKernel {
  std::shared_ptr<void> lib;    // the loaded cubin; unloaded when its last holder lets go
  cudaKernel_t fn = nullptr;
  int block = 128;              // threads per block the source was generated for
  double compile_ms = 0.0;
  bool from_cache = false;      // the cubin came from the disk cache
  bool failed = false;
  std::string error;
};

struct JitState {
  std::mutex mu;
  int device = -1;
  JitKernel k[kKinds];
  int last_used = 0;
};

JitState* jit_state(tami_diagram* d) {
  std::lock_guard<std::mutex> lk(g_jit_mu);
  if (!d->jit) d->jit = new JitState;
  return static_cast<JitState*>(d->jit);
}

void jit_release(tami_diagram* d) {
  if (!d || !d->jit) return;
  delete static_cast<JitState*>(d->jit);
  d->jit = nullptr;
}

// Compile (once per diagram, kind and device) the specialised kernel of d's table.
int jit_prepare(tami_diagram* d, int kind) {
  std::string why;
  if (!jit_supported(d->hdr, kind, &why)) { set_error("specialised kernel: " + why); return TAMI_EUNSUPPORTED; }
  JitState* s = jit_state(d);
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->device != d->device) {          // a new upload device: build again for it
    for (JitKernel& k : s->k) k = JitKernel{};
    s->device = d->device;
  }
  JitKernel& K = s->k[kind];
  if (K.fn) return TAMI_OK;
  if (K.failed) { set_error(K.error); return TAMI_EUNSUPPORTED; }
  auto fail = [&](const std::string& m) {
    K.failed = true;
    K.error = "specialised kernel: " + m;
    set_error(K.error);
    return TAMI_EUNSUPPORTED;
  };
  Nvrtc& nv = nvrtc();
  if (!nv.ok) return fail(nv.why);
  const auto t0 = std::chrono::steady_clock::now();
  const std::string src = jit_source(d->hdr, d->blob.data(), kind);
  K.block = lockstep_block(d->hdr, kind);
  const char* hdr_src[1] = {kDevmathSource};
  const char* hdr_name[1] = {"tami_devmath.cuh"};
  const char* opts[] = {"-arch=sm_103a", "-std=c++17", "-w"};
  const int n_opts = (int)(sizeof opts / sizeof opts[0]);
  // identity of the compilation: compiler, options, the included header and the source
  std::string ident = nv.version + "\n";
  for (const char* o : opts) ident += std::string(o) + " ";
  ident += "\n";
  ident += kDevmathSource;
  ident += "\n";
  ident += src;
  std::string path;
  const std::string dir = jit_cache_dir();
  if (!dir.empty()) {
    char name[32];
    std::snprintf(name, sizeof name, "%016llx.tjc",
                  (unsigned long long)jit_fnv1a(ident.data(), ident.size(), 1469598103934665603ull));
    path = dir + "/" + name;
  }
  auto compile = [&](std::vector<char>* cubin) -> std::string {   // "" on success, else the error
    void* prog = nullptr;
    int rc = nv.create(&prog, src.c_str(), "tami_jit.cu", 1, hdr_src, hdr_name);
    if (rc) return std::string("nvrtcCreateProgram: ") + nv.err(rc);
    rc = nv.compile(prog, n_opts, opts);
    if (rc) {
      size_t n = 0;
      nv.log_size(prog, &n);
      std::string log(n, '\0');
      if (n) nv.log(prog, &log[0]);
      nv.destroy(&prog);
      return std::string("NVRTC compile failed: ") + nv.err(rc) + "\n" + log.substr(0, 2000);
    }
    size_t nb = 0;
    nv.cubin_size(prog, &nb);
    cubin->resize(nb);
    nv.cubin(prog, cubin->data());
    nv.destroy(&prog);
    return "";
  };
  auto load = [&](const std::vector<char>& cubin, std::string* err) {
    cudaLibrary_t lib = nullptr;
    cudaError_t e = cudaLibraryLoadData(&lib, cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) { *err = std::string("cudaLibraryLoadData: ") + cudaGetErrorString(e); return false; }
    K.lib = std::shared_ptr<void>(lib, [](void* l) { cudaLibraryUnload(static_cast<cudaLibrary_t>(l)); });
    e = cudaLibraryGetKernel(&K.fn, lib, kKernelName[kind]);
    if (e != cudaSuccess) {
      K.lib.reset();
      K.fn = nullptr;
      *err = std::string("cudaLibraryGetKernel: ") + cudaGetErrorString(e);
      return false;
    }
    return true;
  };
  std::vector<char> cubin;
  std::string err;
  K.from_cache = !path.empty() && jit_cache_read(path, ident, &cubin) && load(cubin, &err);
  if (!K.from_cache) {
    err = compile(&cubin);
    if (!err.empty()) return fail(err);
    if (!load(cubin, &err)) return fail(err);
    if (!path.empty()) jit_cache_write(path, ident, cubin);   // best effort: a failed write only costs a compile
  }
  K.compile_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return TAMI_OK;
}

// Whether an evaluating call of this kind takes the specialised kernel for n samples (compiling it if
// so): 1 = use it, 0 = the generic kernel, or -status (the "always" mode when it cannot be built).
size_t jit_smem(const TableHeader& h, int kind, int n_f, int block) {
  if (kind == kKindEnergy) return sizeof(double) * (size_t)(2 * h.n_xk + 2 * h.n_cden) * n_f;
  const size_t red = (size_t)block;   // the block reduction's [warp][32] buffer
  const bool adj = kind == kKindFused || kind == kKindBwd;
  const size_t jsv = smem_loop_values(h, adj, block) ? (size_t)block * loop_value_count(h) : 0;
  return sizeof(double) * ((size_t)(4 + 2 * h.n_cden) * n_f + red + jsv);
}

int jit_select(tami_diagram* d, int kind, int64_t n, int n_f, bool generic_ok) {
  const int mode = jit_mode();
  if (mode == TAMI_JIT_NEVER) return 0;
  // large enough to repay a compilation: 2^21 Monte Carlo samples, or 2^25 (row, frequency) values;
  // a table the generic kernel cannot take goes to the specialised one at any size
  const bool big = !generic_ok || (kind == kKindEnergy ? (double)n * n_f >= 33554432.0 : n >= (int64_t(1) << 21));
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, d->device);
  const bool fits = (kind == kKindEnergy || n_f <= kJitMaxFreq) &&
                    jit_smem(d->hdr, kind, n_f, lockstep_block(d->hdr, kind)) <= (size_t)optin;
  if (mode == TAMI_JIT_AUTO && (!big || !fits || !jit_supported(d->hdr, kind, nullptr))) return 0;
  if (!fits) { set_error("specialised kernel: frequencies beyond its per-thread sums or shared memory"); return -TAMI_EUNSUPPORTED; }
  const int rc = jit_prepare(d, kind);
  if (rc == TAMI_OK) return 1;
  return mode == TAMI_JIT_ALWAYS ? -rc : 0;
}

int jit_handle(tami_diagram* d, int kind, int n_f, JitHandle* h) {
  const int rc = jit_prepare(d, kind);
  if (rc) return rc;
  JitState* s = jit_state(d);
  std::lock_guard<std::mutex> lk(s->mu);
  h->lib = s->k[kind].lib;
  h->fn = reinterpret_cast<void*>(s->k[kind].fn);
  h->block = s->k[kind].block;
  h->smem = jit_smem(d->hdr, kind, n_f, h->block);
  return TAMI_OK;
}

int jit_grid(const JitHandle& h, int64_t n, int max_grid, int* grid_out) {
  cudaError_t e = cudaFuncSetAttribute(h.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h.smem);
  if (e != cudaSuccess) { set_error(std::string("specialised kernel attribute: ") + cudaGetErrorString(e)); return TAMI_ECUDA; }
  int per_sm = 0, sms = 0, dev = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, h.fn, h.block, h.smem) != cudaSuccess || per_sm < 1) per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = (long long)sms * per_sm;
  const long long tiles = (n + h.block - 1) / h.block;
  if (grid > tiles) grid = tiles;
  if (grid > max_grid) grid = max_grid;   // the caller's workspace holds max_grid partial rows
  if (grid < 1) grid = 1;
  *grid_out = (int)grid;
  return TAMI_OK;
}

int jit_launch_at(const JitHandle& h, int grid, const tami_lattice* lat, const double* params, uint64_t seed,
                  uint64_t offset, int64_t n, const double* X, int n_f, double beta, const double* gout,
                  double* per_sample, double* ps_dX, double* ps_grad, double* saved, double* partial,
                  struct CUstream_st* st) {
  double lt = lat ? lat->t : 0.0, ltp = lat ? lat->tp : 0.0, lmu = lat ? lat->mu : 0.0;
  double lkx = lat ? lat->kx_ext : 0.0, lky = lat ? lat->ky_ext : 0.0;
  unsigned long long sd = seed, off = offset;
  long long nn = n;
  int nf = n_f;
  double b = beta;
  const double *Xp = X, *Gp = gout, *Pp = params;
  double *pdx = ps_dX, *pg = ps_grad, *pv = per_sample, *sv = saved, *pp = partial;
  void* args[] = {&lt, &ltp, &lmu, &lkx, &lky, &sd, &off, &nn, &Xp, &Gp, &nf, &b, &pdx, &pg, &pv, &sv, &pp, &Pp};
  const cudaError_t e = cudaLaunchKernel(h.fn, dim3((unsigned)grid), dim3((unsigned)h.block), args, h.smem, st);
  if (e != cudaSuccess) { set_error(std::string("specialised kernel launch: ") + cudaGetErrorString(e)); return TAMI_ECUDA; }
  return TAMI_OK;
}

int jit_launch(tami_diagram* d, int kind, const tami_lattice* lat, uint64_t seed, uint64_t offset, int64_t n,
               const double* X, int n_f, double beta, const double* gout, double* per_sample, double* ps_dX,
               double* ps_grad, double* saved, double* partial, int max_grid, struct CUstream_st* st, int* grid_out) {
  JitHandle h;
  int rc = jit_handle(d, kind, n_f, &h);
  if (!rc) rc = jit_grid(h, n, max_grid, grid_out);
  if (!rc) rc = jit_launch_at(h, *grid_out, lat, nullptr, seed, offset, n, X, n_f, beta, gout, per_sample, ps_dX,
                              ps_grad, saved, partial, st);
  if (rc) return rc;
  jit_state(d)->last_used = 1;
  return TAMI_OK;
}

int jit_select_batch(tami_diagram* const* ds, int n_d, const int64_t* n, int n_f, int* use) {
  for (int d = 0; d < n_d; ++d) use[d] = 0;
  const int mode = jit_mode();
  if (mode == TAMI_JIT_NEVER) return TAMI_OK;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  std::vector<int> todo;
  for (int d = 0; d < n_d; ++d) {
    std::string why;
    const bool fits = n_f <= kJitMaxFreq && jit_smem(ds[d]->hdr, kKindFwd, n_f, lockstep_block(ds[d]->hdr, kKindFwd)) <= (size_t)optin;
    const bool ok = fits && jit_supported(ds[d]->hdr, kKindFwd, &why);
    if (mode == TAMI_JIT_AUTO && (n[d] < (int64_t(1) << 20) || !ok)) continue;
    if (!ok) {
      set_error("specialised kernel: " + (fits ? why : std::string("frequencies beyond its per-thread sums or shared memory")));
      return TAMI_EUNSUPPORTED;
    }
    todo.push_back(d);
  }
  // compile on up to one host thread per core (NVRTC programs are independent)
  std::vector<int> rc(todo.size(), TAMI_OK);
  std::vector<std::string> err(todo.size());
  std::atomic<size_t> next{0};
  auto work = [&]() {
    cudaSetDevice(dev);
    for (size_t i; (i = next.fetch_add(1)) < todo.size();) {
      rc[i] = jit_prepare(ds[todo[i]], kKindFwd);
      if (rc[i]) err[i] = tami_last_error();
    }
  };
  const size_t n_thr = std::min<size_t>(std::max(1u, std::thread::hardware_concurrency()), todo.size());
  std::vector<std::thread> pool;
  for (size_t t = 1; t < n_thr; ++t) {
    try {
      pool.emplace_back(work);
    } catch (...) {            // no more threads to be had: the ones running (and this one) finish the list
      break;
    }
  }
  work();
  for (std::thread& t : pool) t.join();
  for (size_t i = 0; i < todo.size(); ++i) {
    if (rc[i] == TAMI_OK) {
      use[todo[i]] = 1;
    } else if (mode == TAMI_JIT_ALWAYS) {
      set_error(err[i]);
      return rc[i];
    }
  }
  return TAMI_OK;
}

void jit_mark_generic(tami_diagram* d) {
  if (d->jit) static_cast<JitState*>(d->jit)->last_used = 0;
}

}  // namespace tami

using namespace tami;

extern "C" {

int tami_set_jit(int mode) {
  if (mode < TAMI_JIT_NEVER || mode > TAMI_JIT_ALWAYS) { set_error("mode must be 0, 1 or 2"); return TAMI_EINVAL; }
  std::lock_guard<std::mutex> lk(g_jit_mu);
  g_jit_mode = mode;
  return TAMI_OK;
}

int tami_jit_prepare(tami_diagram* d) {
  return guarded([&]() -> int {
  if (!d) { set_error("NULL diagram"); return TAMI_EINVAL; }
  if (!d->d_blob) { set_error("diagram not uploaded (call tami_upload)"); return TAMI_EINVAL; }
  int built = 0;
  for (int k = 0; k < kKinds; ++k) {
    if (!jit_supported(d->hdr, k, nullptr)) continue;
    const int rc = jit_prepare(d, k);
    if (rc) return rc;
    ++built;
  }
  if (!built) { set_error("specialised kernel: no kind applies to this table"); return TAMI_EUNSUPPORTED; }
  return TAMI_OK;
  });
}

int tami_jit_cached(const tami_diagram* d, int* from_cache) {
  if (!d || !from_cache) { set_error("NULL argument"); return TAMI_EINVAL; }
  const JitState* s = static_cast<const JitState*>(d->jit);
  int mask = 0;
  if (s)
    for (int k = 0; k < kKinds; ++k)
      if (s->k[k].fn && s->k[k].from_cache) mask |= 1 << k;
  *from_cache = mask;
  return TAMI_OK;
}

int tami_jit_status(const tami_diagram* d, int* ready, int* last_used, double* compile_ms) {
  if (!d) { set_error("NULL diagram"); return TAMI_EINVAL; }
  const JitState* s = static_cast<const JitState*>(d->jit);
  int mask = 0;
  double ms = 0.0;
  if (s)
    for (int k = 0; k < kKinds; ++k)
      if (s->k[k].fn) { mask |= 1 << k; ms += s->k[k].compile_ms; }
  if (ready) *ready = mask;
  if (last_used) *last_used = s ? s->last_used : 0;
  if (compile_ms) *compile_ms = ms;
  return TAMI_OK;
}

int tami_jit_source(const tami_diagram* d, int kind, char* buf, size_t cap, size_t* len) {
  return guarded([&]() -> int {
  if (!d) { set_error("NULL diagram"); return TAMI_EINVAL; }
  if (kind < 0 || kind >= kKinds) {
    set_error("kind must be 0 (fused), 1 (forward), 2 (adjoint) or 3 (energy input)");
    return TAMI_EINVAL;
  }
  std::string why;
  if (!jit_supported(d->hdr, kind, &why)) { set_error("specialised kernel: " + why); return TAMI_EUNSUPPORTED; }
  const std::string src = jit_source(d->hdr, d->blob.data(), kind);
  if (len) *len = src.size() + 1;
  if (buf && cap > 0) {
    const size_t k = std::min(cap - 1, src.size());
    std::memcpy(buf, src.data(), k);
    buf[k] = '\0';
  }
  return TAMI_OK;
  });
}

}  // extern "C"
