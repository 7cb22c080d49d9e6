// Device arithmetic of the libtami kernels: the counter-based momentum sampler, the lattice
// dispersion with its Cody-Waite cos/sin, the table-driven exponential, the reciprocal and the
// Fermi/Bose values and derivatives of one table segment.  Self-contained (no host headers, plain
// integer types), so that the same text also serves the kernels the library generates and
// compiles at run time for one diagram's table (tami_jit.cpp).  Internal to the library.
#pragma once

namespace tami {
namespace dev {

constexpr int kBlock = 128;                 // threads per block = samples per tile

__device__ __forceinline__ void philox4x32_10(unsigned int c[4], unsigned int k0, unsigned int k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    unsigned int hi0 = __umulhi(0xD2511F53u, c[0]), lo0 = 0xD2511F53u * c[0];
    unsigned int hi1 = __umulhi(0xCD9E8D57u, c[2]), lo1 = 0xCD9E8D57u * c[2];
    unsigned int n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    k0 += 0x9E3779B9u; k1 += 0xBB67AE85u;
  }
}

// [0,1) from 53 bits of two words, u = m 2^-53, then k = 2 pi u - pi with one rounding.  m is
// exact in a double and the powers of two scale exactly, so fma(m, 2 pi 2^-53, -pi) is that
// rounding of the same real number: one FP64 multiply fewer.
__device__ __forceinline__ double to_momentum(unsigned int hi, unsigned int lo) {
  unsigned long long m = ((unsigned long long)hi << 21) | (unsigned long long)(lo >> 11);
  const double pi = 0x1.921fb54442d18p+1;
  return fma(__ull2double_rn(m), 2.0 * pi * 0x1.0p-53, -pi);
}

// ---------------------------------------------------------------------------------------------
// Double-precision multiplication on the integer pipes.  On this GPU the FP64 unit is the
// bottleneck of the evaluation kernels while the integer units sit mostly idle, and the two run
// concurrently.  imul computes the IEEE round-to-nearest-even product of two doubles with 64-bit
// integer arithmetic, bit for bit what DMUL gives, so a kernel can move part of its FP64 work to
// the integer pipes.  The integer fast path covers normal operands with a normal result; zeros,
// subnormals, infinities, NaNs and results that would underflow or overflow take the FP64
// instruction instead, out of line, so that the fast path issues no FP64 instruction at all.
// (Textbook IEEE 754 multiplication: the exact 106-bit product of the significands, normalised,
// rounded to nearest even with round and sticky bits.)
static __device__ __noinline__ double dmul_fp64(double a, double b) { return __dmul_rn(a, b); }

// The normal path shared by imul and imul_ftz: the rounded product's bits for normal operands
// whose result is normal (e in [1, 0x7FE]); e, the biased exponent before rounding, says whether
// it is.
__device__ __forceinline__ unsigned long long imul_bits(unsigned long long ua, unsigned long long ub, int ea, int eb,
                                                        int& e) {
  const unsigned long long sign = (ua ^ ub) & 0x8000000000000000ull;
  const unsigned long long ma = (ua & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const unsigned long long mb = (ub & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
  const unsigned long long lo = ma * mb, hi = __umul64hi(ma, mb);   // 106-bit product in [2^104, 2^106)
  const int top = (int)(hi >> 41);                                   // 1: bit 105 is set
  const unsigned long long t = (hi << (23 - top)) | (lo >> (41 + top));   // leading one at bit 63
  const unsigned long long below = lo << (23 - top);                // product bits under t
  unsigned long long m = t >> 11;                                    // 53 significant bits
  const unsigned long long rb = (t >> 10) & 1ull;
  const unsigned long long st = ((t & 0x3FFull) | below) != 0ull;
  m += rb & (st | (m & 1ull));                                       // may carry into bit 53
  e = ea + eb - 1023 + top;
  return sign | (((unsigned long long)(e - 1) << 52) + m);
}

__device__ __forceinline__ double imul(double a, double b) {
  const unsigned long long ua = __double_as_longlong(a), ub = __double_as_longlong(b);
  const int ea = (int)(ua >> 52) & 0x7FF, eb = (int)(ub >> 52) & 0x7FF;
  int e;
  const unsigned long long r = imul_bits(ua, ub, ea, eb, e);
  if (ea == 0 || eb == 0 || ea == 0x7FF || eb == 0x7FF || e <= 0 || e >= 0x7FE) return dmul_fp64(a, b);
  return __longlong_as_double(r);
}

// The same product without the FP64 instruction anywhere (no call, no branch: the compiler cannot
// turn it into a predicated DMUL that would take an FP64 issue slot), for code whose products all
// move to the integer pipes.  Normal operands with a normal result: the IEEE product, bit for bit.
// Otherwise flush to zero: a zero or subnormal operand, or a result below the normal range, gives
// a signed zero; a result above the range a signed infinity; an infinite operand a signed
// infinity (a NaN against a zero or subnormal one); a NaN operand a quiet NaN (its payload kept).
__device__ __forceinline__ double imul_ftz(double a, double b) {
  const unsigned long long ua = __double_as_longlong(a), ub = __double_as_longlong(b);
  const int ea = (int)(ua >> 52) & 0x7FF, eb = (int)(ub >> 52) & 0x7FF;
  int e;
  unsigned long long r = imul_bits(ua, ub, ea, eb, e);
  const unsigned long long sign = (ua ^ ub) & 0x8000000000000000ull;
  const bool zero_in = ea == 0 || eb == 0;
  r = (e <= 0 || zero_in) ? sign : r;
  r = (e >= 0x7FF && !zero_in) ? (sign | 0x7FF0000000000000ull) : r;
  const bool a_nan = (ua << 1) > 0xFFE0000000000000ull, b_nan = (ub << 1) > 0xFFE0000000000000ull;
  const bool inf_in = ea == 0x7FF || eb == 0x7FF;
  const unsigned long long special = a_nan ? (ua | 0x0008000000000000ull)
                                   : b_nan ? (ub | 0x0008000000000000ull)
                                   : zero_in ? 0x7FF8000000000000ull : (sign | 0x7FF0000000000000ull);
  r = inf_in ? special : r;
  return __longlong_as_double(r);
}


// cos and sin: Cody-Waite reduction by pi (two-part constant), k = n pi + r, |r| <= pi/2 (n the
// integer nearest to k/pi, from one fma against 1.5 * 2^52), then
// Taylor series in r (to r^20 for cos, r^21 for sin) and the sign (-1)^n (W. J. Cody and
// W. Waite, 1980).  Every operation is an explicit fma or a rounded mul intrinsic, so the result
// is the same on any IEEE machine that follows the same recipe.
// n = nearest integer to k/pi, read from the low word of k/pi + 1.5 * 2^52 (one rounding);
// r = k - n pi with the first two parts of a three-part pi (the third, times n, lies below the
// rounding for the momenta the lattice produces); odd = n & 1.
__device__ __forceinline__ double cw_reduce(double k, int& odd) {
  const double inv_pi = 0x1.45f306dc9c883p-2;
  const double P1 = 0x1.921fb54442d18p+1, P2 = 0x1.1a62633145c07p-53;
  const double nd = fma(k, inv_pi, 0x1.8p52);
  odd = __double2loint(nd) & 1;
  const double n = nd - 0x1.8p52;
  const double r = fma(-n, P1, k);      // exact: k - n P1 is a multiple of 2^-52 below 2 in magnitude
  return fma(-n, P2, r);                // n P3 < 3e-32 for |k| < 22 is below the rounding
}

__device__ __forceinline__ double flip_if(double v, int odd) {   // (-1)^odd v, on the sign bit
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)odd << 63));
}

__device__ __forceinline__ double cw_cos_poly(double z) {
  double pc = 0x1.e542ba4020225p-62;
  pc = fma(pc, z, -0x1.6827863b97d97p-53);
  pc = fma(pc, z, 0x1.ae7f3e733b81fp-45);
  pc = fma(pc, z, -0x1.93974a8c07c9dp-37);
  pc = fma(pc, z, 0x1.1eed8eff8d898p-29);
  pc = fma(pc, z, -0x1.27e4fb7789f5cp-22);
  pc = fma(pc, z, 0x1.a01a01a01a01ap-16);
  pc = fma(pc, z, -0x1.6c16c16c16c17p-10);
  pc = fma(pc, z, 0x1.5555555555555p-5);
  pc = fma(pc, z, -0x1.0000000000000p-1);
  return fma(z, pc, 1.0);
}

__device__ __forceinline__ double cw_cos(double k) {
  int odd;
  const double r = cw_reduce(k, odd);
  return flip_if(cw_cos_poly(__dmul_rn(r, r)), odd);
}

__device__ __forceinline__ void cw_sincos(double k, double& s_out, double& c_out) {
  int odd;
  const double r = cw_reduce(k, odd);
  const double z = __dmul_rn(r, r);
  const double cr = cw_cos_poly(z);
  double ps = 0x1.71b8ef6dcf572p-66;
  ps = fma(ps, z, -0x1.2f49b46814157p-57);
  ps = fma(ps, z, 0x1.952c77030ad4ap-49);
  ps = fma(ps, z, -0x1.ae7f3e733b81fp-41);
  ps = fma(ps, z, 0x1.6124613a86d09p-33);
  ps = fma(ps, z, -0x1.ae64567f544e4p-26);
  ps = fma(ps, z, 0x1.71de3a556c734p-19);
  ps = fma(ps, z, -0x1.a01a01a01a01ap-13);
  ps = fma(ps, z, 0x1.1111111111111p-7);
  ps = fma(ps, z, -0x1.5555555555555p-3);
  const double sr = fma(__dmul_rn(r, z), ps, r);
  s_out = flip_if(sr, odd);
  c_out = flip_if(cr, odd);
}

// E = mu - eps(k),  eps(k) = -2t(cos kx + cos ky) - 4t' cos kx cos ky
__device__ __forceinline__ double line_energy(double kx, double ky, double t, double tp, double mu) {
  const double cx = cw_cos(kx), cy = cw_cos(ky);
  const double sum = __dadd_rn(cx, cy);
  const double prod = __dmul_rn(cx, cy);
  return fma(4.0 * tp, prod, fma(2.0 * t, sum, mu));
}

// Energy of a line that carries k_ext, with the factors G = (2t + 4t' cos K_perp) sin K of
// dE/dK = -G for both components (one sincos per component); E has line_energy's bits.
__device__ __forceinline__ double line_energy_grad(double kx, double ky, double t, double tp, double mu, double& gx,
                                                   double& gy) {
  double sx, cx, sy, cy;
  cw_sincos(kx, sx, cx);
  cw_sincos(ky, sy, cy);
  gx = fma(4.0 * tp, cy, 2.0 * t) * sx;
  gy = fma(4.0 * tp, cx, 2.0 * t) * sy;
  return fma(4.0 * tp, __dmul_rn(cx, cy), fma(2.0 * t, __dadd_rn(cx, cy), mu));
}

// e^t and e^t - 1 for t <= 0, after P. T. P. Tang, "Table-driven implementation of the exponential
// function in IEEE floating-point arithmetic", ACM TOMS 15 (1989) 144-157:
// t = k ln2/32 + r with k = 32 m + j (0 <= j < 32), |r| <= ln2/64, and
// e^t = 2^m 2^(j/32) e^r, 2^(j/32) = T_hi + T_lo from a two-part table, e^r - 1 = p(r) its Taylor
// polynomial to r^7 (truncation < 4e-19 relative).  k is read from the low word of
// t * 32/ln2 + 1.5 * 2^52 (round to nearest), and r is formed with a two-part ln2/32 whose high
// part has few enough bits that the first reduction step is exact.  Then
//   e^t     = T_hi' + (T_hi' p + T_lo'),        e^t - 1 = (T_hi' - 1) + (T_hi' p + T_lo'),
// T' = 2^m T; T_hi' - 1 is exact where it matters (T_hi' in [1/2, 1]).  Without e^t - 1 the sum is
// formed unscaled, T_hi + (T_hi p + T_lo) in [1/2, 2), and scaled by 2^m with an exponent add
// (exact, so the same bits as scaling first).
__device__ const double kExp2TabHi[32] = {
  0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0,
  0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, 0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0,
  0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
  0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0,
  0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, 0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0,
  0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
  0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0,
  0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, 0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0};
__device__ const double kExp2TabLo[32] = {
  0x0.0p+0, 0x1.d73e2a475b465p-55, 0x1.8a62e4adc610bp-54, -0x1.6c51039449b3ap-54,
  -0x1.19041b9d78a76p-55, 0x1.e016e00a2643cp-54, 0x1.9b07eb6c70573p-54, 0x1.612e8afad1255p-55,
  0x1.6f46ad23182e4p-55, -0x1.63aeabf42eae2p-54, 0x1.ada0911f09ebcp-55, 0x1.89b7a04ef80d0p-59,
  0x1.d4397afec42e2p-56, -0x1.07abe1db13cadp-55, 0x1.6324c054647adp-54, -0x1.383c17e40b497p-54,
  -0x1.bdd3413b26456p-54, -0x1.16e4786887a99p-55, -0x1.41577ee04992fp-55, -0x1.d4c1dd41532d8p-54,
  0x1.6e9f156864b27p-54, -0x1.75fc781b57ebcp-57, 0x1.c7c46b071f2bep-56, -0x1.d2f6edb8d41e1p-54,
  0x1.7a1cd345dcc81p-54, -0x1.5584f7e54ac3bp-56, 0x1.11065895048ddp-55, 0x1.503cbd1e949dbp-56,
  0x1.2ed02d75b3707p-55, -0x1.1a5cd4f184b5cp-54, -0x1.e9c23179c2893p-54, 0x1.9d3e12dd8a18bp-54};

// 2^m T_hi (1 + p) for m < -960 (T_lo dropped), with 2^m applied in two steps; 0 below 2^-2000.
// Out of line so that the common path carries no predicated FP64 work.
static __device__ __noinline__ double exp_neg_deep_tail(double th, double p, int m) {
  if (m < -2000) return 0.0;
  th = __longlong_as_double(__double_as_longlong(th) + ((long long)(m + 1000) << 52));
  return fma(th, p, th) * 0x1.0p-1000;
}

template <bool NEED_EM>
__device__ __forceinline__ double exp_neg(double t, double& em) {
  const double kd = fma(t, 0x1.71547652b82fep+5, 0x1.8p52);
  const int k = __double2loint(kd);
  const double kf = kd - 0x1.8p52;
  double r = fma(-kf, 0x1.62e42fefa4000p-6, t);
  r = fma(-kf, -0x1.8432a1b0e2634p-48, r);
  const double r2 = r * r;
  double q = 0x1.a01a01a01a01ap-13;
  q = fma(q, r, 0x1.6c16c16c16c17p-10);
  q = fma(q, r, 0x1.1111111111111p-7);
  q = fma(q, r, 0x1.5555555555555p-5);
  q = fma(q, r, 0x1.5555555555555p-3);
  q = fma(q, r, 0x1.0000000000000p-1);
  const double p = fma(r2, q, r);                 // e^r - 1
  const int j = k & 31, m = k >> 5;
  double th = __ldg(&kExp2TabHi[j]), tl = __ldg(&kExp2TabLo[j]);
  double y;
  if (m >= -960) {                                 // 2^m T_hi and 2^m T_lo stay normal numbers
    const long long sh = (long long)m << 52;
    if (NEED_EM) {
      th = __longlong_as_double(__double_as_longlong(th) + sh);
      // only the j = 0 entry of the low table is 0 (kept 0 rather than exponent-shifted); an
      // integer test, not an FP64 compare
      tl = j == 0 ? 0.0 : __longlong_as_double(__double_as_longlong(tl) + sh);
      const double c = fma(th, p, tl);
      y = th + c;
      em = (th - 1.0) + c;
    } else {
      y = __longlong_as_double(__double_as_longlong(th + fma(th, p, tl)) + sh);
    }
  } else {
    y = exp_neg_deep_tail(th, p, m);               // e^t < 1e-289: a real branch, rarely taken
    if (NEED_EM) em = y - 1.0;
  }
  return y;
}

// 1/d: hardware estimate refined by one third-order Newton-Raphson step,
// r <- r (1 + e + e^2), e = 1 - d r  (error e^3).
__device__ __forceinline__ double rcp(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
  double e = fma(-d, r, 1.0);
  return fma(r, fma(e, e, e), r);
}

// d^k/dx^k g at (g, h = 1 - g): (-beta)^k sum_i (-1)^i A(k,i) g^(i+1) h^(k-i), A = Eulerian
// Out of line: derivative values are few per sample, and one copy keeps the kernels' code small
// (instruction-fetch stalls are measurable in the adjoint).
static __device__ __noinline__ double fermi_poly(int k, double g, double h, double beta) {
  if (k == 0) return g;
  double gh = g * h;
  if (k == 1) return -beta * gh;
  double d = h - g;
  if (k == 2) return beta * beta * gh * d;
  if (k == 3) return -beta * beta * beta * gh * fma(d, d, -2.0 * gh);
  double b4 = beta * beta * beta * beta;
  double h2 = h * h, g2 = g * g;
  if (k == 4) return b4 * gh * (h2 * h - 11.0 * g * h2 + 11.0 * g2 * h - g2 * g);
  return -b4 * beta * gh * (h2 * h2 - 26.0 * g * h2 * h + 66.0 * g2 * h2 - 26.0 * g2 * g * h + g2 * g2);
}

// Fermi values of one segment of the term table: one energy combination x and one sigma, every
// value g_sigma^(k)(+-x) that the terms use (k = 0 first).  y = e^{-beta|x|} keeps the tails exact;
// the Bose-type segments (sigma = -1) take 1 - y = -(e^t - 1) from the same exponential.  With
// DUAL, fvd holds each value's derivative with respect to its own argument (order k + 1).
// seg = {combo, sigma, v_begin, first v with k >= 1, v_end}; fvr[v] = {sign, k}.
template <bool BOSE, bool DUAL>
__device__ __forceinline__ void fermi_segment(const int* seg, const int* fvr, const double* x, double beta,
                                              double* fv, double* fvd) {
  const double xv = x[seg[0]];
  double em = 0.0;
  const double y = exp_neg<BOSE>(-beta * fabs(xv), em);
  const double rD = rcp(BOSE ? -em : 1.0 + y);
  const double t2 = (BOSE ? -y : y) * rD;
  const bool neg = __double_as_longlong(xv) <= 0;   // xv <= 0 (+0, -0 and negatives), on the ALU
  const double g = neg ? rD : t2, h = neg ? t2 : rD;   // g_sigma(x) and g_sigma(-x)
  double d1 = 0.0;
  if (DUAL) d1 = -beta * (g * h);
  for (int v = seg[2]; v < seg[3]; ++v) {
    fv[v] = fvr[2 * v] > 0 ? g : h;
    if (DUAL) fvd[v] = d1;
  }
  for (int v = seg[3]; v < seg[4]; ++v) {
    const bool pos = fvr[2 * v] > 0;
    const int k = fvr[2 * v + 1];
    const double gg = pos ? g : h, hg = pos ? h : g;
    fv[v] = fermi_poly(k, gg, hg, beta);
    if (DUAL) fvd[v] = fermi_poly(k + 1, gg, hg, beta);
  }
}

}  // namespace dev
}  // namespace tami
