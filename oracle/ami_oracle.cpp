// ORACLE -- test infrastructure only.
//
// A plain, slow, obviously-correct FP64 CPU restatement of algorithmic Matsubara
// integration (AMI) as described in "TorchAmi: Generalized CPU/GPU Implementation of
// Algorithmic Matsubara Integration" (Burke & LeBlanc, arXiv:2311.17189).  It exists to
// check the CUDA path; only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
// leg may load it.  It shares no code, header, table or constant generator with the
// library under paper_2311_17189_gb300/, and the library never loads it.
//
// What it computes (paper section in brackets):
//   * construction [Sec. 2.2, Eqs. goal, Green_Function, Res_Th, Poles, Res_mul]: the
//     integrand beta^-m sum_{nu} prod_j 1/(X_j + E_j) is summed one internal frequency at a
//     time by the residue theorem, with multipole residues through the Leibniz rule; every
//     resulting term is A * prod(Fermi/Bose factors) * prod(Green's functions)
//     [Sec. 2.2, "I = A FT R"], kept flat (the FACTORIZE=false form);
//   * evaluation [Sec. 2.3]: terms evaluated one by one for a batch of energies and
//     rows of external frequencies (n_ext >= 1 external variables, the last columns of the
//     labels, as in the frequency_t rows of Sec. 2.3), summed with Neumaier compensation;
//   * momentum sampling [Sec. 5.2]: K = k A^T line momenta and a per-line dispersion;
//   * forward-mode dual-number derivatives of the same evaluation (d/d omega, d/d mu,
//     d/d k_ext) -- an independent check of an adjoint;
//   * brute-force truncated Matsubara sums (the plain definition, Eq. goal);
//   * a brute-force Wick enumerator of Hubbard self-energy diagrams with a momentum
//     labeller [Sec. 2.5 describes graph input and labelling].
//
// Readings of the paper that the text leaves open:
//   R1  pole of G_j in nu_p: the root of alpha_p^j z + rest = 0, i.e.
//       z = -alpha_p^j (E_j + sum_{l!=p} i alpha_l^j nu_l) for alpha_p^j = +-1 (Eq. Poles
//       prints the inner energy with the dispersion's sign).
//   R2  Bosonic internal variables use -n_B as the residue weight (standard bosonic sum);
//       the paper states only the fermionic theorem (Eq. Res_Th).
//   R3  Fermi/Bose factors carrying a Matsubara shift S are reduced by periodicity:
//       f(x+iS) = -n_B(x) and -n_B(x+iS) = f(x) for fermionic S, unchanged for bosonic S,
//       which makes FT frequency independent (Sec. 2.2 states FT does not depend on nu).
//       g_sigma(x) = 1/(sigma e^{beta x} + 1): sigma=+1 is f, sigma=-1 is -n_B.
//   R4  |alpha_p| > 1 in a summed variable is rejected; E_REG is fixed to 0.
//   R5  identical Green's functions (equal energy and frequency coefficients) are grouped
//       into powers before each residue step; the multipole residue is expanded with the
//       Leibniz rule over the distinct factors, and no terms are merged afterwards.
//
// Inputs.  Philox momenta and the u -> k map are integer and one-rounding operations, line
// momenta are sums of the labelled momenta in variable order, and the dispersion is the plain
// definition with the C library's cos and sin (the paper leaves the dispersion eps(k) to the
// user, Sec. 5.2).  An independent device implementation therefore sees the same momenta bit
// for bit and energies that differ by the two sides' trig and rounding errors; the per-sample
// sensitivity sum_t sum_j |d term_t / d E_j| returned with each evaluation bounds what such an
// energy difference can change.  Compile with -ffp-contract=off.
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <map>
#include <set>
#include <string>
#include <thread>
#include <vector>

using cplx = std::complex<double>;

namespace {

std::string g_err;
int fail(const std::string& m) { g_err = m; return -1; }

// ---------------------------------------------------------------------------------------
// Philox4x32-10 (J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
// numbers: as easy as 1, 2, 3", SC'11).  Ten rounds; the key is bumped by the Weyl
// constants before every round but the first.
// ---------------------------------------------------------------------------------------
void philox(const uint32_t in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c[4] = {in[0], in[1], in[2], in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
    uint32_t n1 = (uint32_t)p1;
    uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
    uint32_t n3 = (uint32_t)p0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
  }
  for (int i = 0; i < 4; ++i) out[i] = c[i];
}

// Uniform double in [0,1) from two 32-bit words: 53 bits (hi word on top) times 2^-53.
double unit53(uint32_t hi, uint32_t lo) {
  uint64_t m = ((uint64_t)hi << 21) | (uint64_t)(lo >> 11);
  return (double)m * 0x1.0p-53;
}

// Momentum component on [-pi, pi): k = 2 pi u - pi with one rounding.
double momentum_from_unit(double u) {
  const double pi = 0x1.921fb54442d18p+1;
  return std::fma(u, 2.0 * pi, -pi);
}

// Sample s, internal momentum l: counter (s_lo, s_hi, l, 0), key (seed_lo, seed_hi); the
// four output words give kx (words 0,1) and ky (words 2,3).
void sample_momentum(uint64_t seed, uint64_t s, int l, double* kx, double* ky) {
  uint32_t ctr[4] = {(uint32_t)s, (uint32_t)(s >> 32), (uint32_t)l, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t w[4];
  philox(ctr, key, w);
  *kx = momentum_from_unit(unit53(w[0], w[1]));
  *ky = momentum_from_unit(unit53(w[2], w[3]));
}

// Hubbard dispersion on the square lattice, eps(k) = -2t(cos kx + cos ky) - 4t' cos kx cos ky;
// the line energy of the integrand is E = mu - eps(k)  (the paper's epsilon^j is minus the
// dispersion, Eq. Green_Function; the chemical potential enters with it).
double line_energy(double kx, double ky, double t, double tp, double mu) {
  double cx = std::cos(kx), cy = std::cos(ky);
  return mu + 2.0 * t * (cx + cy) + 4.0 * tp * cx * cy;
}

// d eps / d kx at (kx, ky): 2t sin kx + 4t' sin kx cos ky.
double deps_dkx(double kx, double ky, double t, double tp) {
  return 2.0 * t * std::sin(kx) + 4.0 * tp * std::sin(kx) * std::cos(ky);
}

// ---------------------------------------------------------------------------------------
// Symbolic objects.
// ---------------------------------------------------------------------------------------
struct GFac {              // 1 / (sum_l i a_l nu_l + sum_j e_j E_j)  (Eq. Green_Function)
  std::vector<int> e;      // energy coefficients over the N base energies
  std::vector<int> a;      // frequency coefficients, the external variables last
  bool operator==(const GFac& o) const { return e == o.e && a == o.a; }
};
struct FFac {              // d^k/dx^k g_sigma(x) at x = c.E
  std::vector<int> c;
  int sigma;
  int k;
};
struct Term {
  double A;
  std::vector<FFac> F;
  std::vector<GFac> G;     // repeated entries are powers
};

struct Solution {
  int N = 0, nv = 0;       // lines (base energies), variables (m internal + n_ext external)
  int n_ext = 1;           // external frequencies, the last n_ext variables (Sec. 2.3)
  std::vector<Term> terms;
  double prefactor = 1.0;
};

double factorial(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }
double binom(int n, int k) {
  double r = 1;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}

// All ways to write n as an ordered sum of `parts` non-negative integers.
void compositions(int n, int parts, std::vector<int>& cur, std::vector<std::vector<int>>& out) {
  if ((int)cur.size() == parts - 1) {
    cur.push_back(n);
    out.push_back(cur);
    cur.pop_back();
    return;
  }
  for (int i = 0; i <= n; ++i) {
    cur.push_back(i);
    compositions(n - i, parts, cur, out);
    cur.pop_back();
  }
}

// One Matsubara sum over variable p of every term (Eqs. Res_Th, Poles, Res_mul).
int sum_variable(const std::vector<Term>& in, int p, bool p_is_boson,
                 const std::vector<int>& var_is_boson, std::vector<Term>& out) {
  out.clear();
  for (const Term& T : in) {
    // distinct Green's functions with their powers (reading R5)
    std::vector<GFac> dist;
    std::vector<int> power;
    for (const GFac& g : T.G) {
      bool found = false;
      for (size_t i = 0; i < dist.size(); ++i)
        if (dist[i] == g) { power[i]++; found = true; break; }
      if (!found) { dist.push_back(g); power.push_back(1); }
    }
    // group the z-dependent ones by pole position (reading R1)
    std::vector<std::vector<int>> pole_members;
    std::vector<std::pair<std::vector<int>, std::vector<int>>> pole_keys;
    int z_degree = 0;
    for (size_t i = 0; i < dist.size(); ++i) {
      int ap = dist[i].a[p];
      if (ap == 0) continue;
      if (ap != 1 && ap != -1) return fail("frequency coefficient with |alpha_p| > 1");
      z_degree += power[i];
      std::vector<int> ke(dist[i].e.size()), ka(dist[i].a.size());
      for (size_t j = 0; j < ke.size(); ++j) ke[j] = -ap * dist[i].e[j];
      for (size_t j = 0; j < ka.size(); ++j) ka[j] = (int)j == p ? 0 : -ap * dist[i].a[j];
      auto key = std::make_pair(ke, ka);
      bool found = false;
      for (size_t q = 0; q < pole_keys.size(); ++q)
        if (pole_keys[q] == key) { pole_members[q].push_back((int)i); found = true; break; }
      if (!found) { pole_keys.push_back(key); pole_members.push_back({(int)i}); }
    }
    if (z_degree < 2) return fail("integrand decays slower than 1/z^2 in a summed variable");

    for (size_t q = 0; q < pole_keys.size(); ++q) {
      const std::vector<int>& mem = pole_members[q];
      int M = 0;
      double pref = 1.0;
      for (int i : mem) {
        M += power[i];
        if (power[i] % 2 == 1 && dist[i].a[p] == -1) pref = -pref;   // prod (1/a_p)^q
      }
      const GFac& gj = dist[mem[0]];
      int ajp = gj.a[p];
      // remaining factors: substituted at z0, z-dependent ones get derivatives
      std::vector<int> others, zdep;
      for (size_t i = 0; i < dist.size(); ++i) {
        if (std::find(mem.begin(), mem.end(), (int)i) != mem.end()) continue;
        others.push_back((int)i);
        if (dist[i].a[p] != 0) zdep.push_back((int)i);
      }
      // Fermi/Bose factor at z0: energy c = -a_jp e_j, shift parity (reading R3)
      FFac nf;
      nf.c.resize(gj.e.size());
      for (size_t j = 0; j < gj.e.size(); ++j) nf.c[j] = -ajp * gj.e[j];
      int shift_parity = 0;
      for (size_t l = 0; l < gj.a.size(); ++l)
        if ((int)l != p && !var_is_boson[l]) shift_parity += std::abs(gj.a[l]);
      int sigma = p_is_boson ? -1 : 1;
      if (shift_parity % 2 == 1) sigma = -sigma;
      nf.sigma = sigma;
      bool czero = std::all_of(nf.c.begin(), nf.c.end(), [](int v) { return v == 0; });
      if (czero && sigma == -1) return fail("Bose factor at zero energy");
      // substituted factors
      std::vector<GFac> sub(dist.size());
      for (int i : others) {
        const GFac& g = dist[i];
        int arp = g.a[p];
        GFac s = g;
        for (size_t j = 0; j < s.e.size(); ++j) s.e[j] = g.e[j] - arp * ajp * gj.e[j];
        for (size_t l = 0; l < s.a.size(); ++l) s.a[l] = g.a[l] - arp * ajp * gj.a[l];
        s.a[p] = 0;
        sub[i] = s;
      }
      // Leibniz expansion of d^{M-1}/dz^{M-1} [w(z) prod_others G^q] / (M-1)!
      std::vector<std::vector<int>> comps;
      std::vector<int> cur;
      compositions(M - 1, 1 + (int)zdep.size(), cur, comps);
      for (const auto& kk : comps) {
        Term nt;
        nt.A = T.A * pref / factorial(kk[0]);
        nt.F = T.F;
        FFac f = nf;
        f.k = kk[0];
        nt.F.push_back(f);
        for (int i : others) {
          int extra = 0;
          auto it = std::find(zdep.begin(), zdep.end(), i);
          if (it != zdep.end()) {
            extra = kk[1 + (it - zdep.begin())];
            int arp = dist[i].a[p];
            double c = binom(power[i] + extra - 1, extra);
            if (extra % 2 == 1) c = -c;                  // (-1)^k
            if (extra % 2 == 1 && arp == -1) c = -c;     // a_rp^k
            nt.A *= c;
          }
          bool zero = std::all_of(sub[i].e.begin(), sub[i].e.end(), [](int v) { return v == 0; }) &&
                      std::all_of(sub[i].a.begin(), sub[i].a.end(), [](int v) { return v == 0; });
          if (zero) return fail("vanishing denominator after substitution");
          for (int r = 0; r < power[i] + extra; ++r) nt.G.push_back(sub[i]);
        }
        out.push_back(nt);
      }
    }
  }
  return 0;
}

int construct(int N, int nv, int n_ext, const int* alpha, const int* eps, const int* boson,
              const int* order, double prefactor, Solution& S) {
  if (N < 1 || n_ext < 1 || nv < n_ext + 1) return fail("bad sizes");
  const int m = nv - n_ext;
  S.N = N;
  S.nv = nv;
  S.n_ext = n_ext;
  S.prefactor = prefactor;
  std::vector<int> vb(nv, 0);
  if (boson) for (int l = 0; l < nv; ++l) vb[l] = boson[l] ? 1 : 0;
  Term t0;
  t0.A = 1.0;
  for (int j = 0; j < N; ++j) {
    GFac g;
    g.a.assign(alpha + j * nv, alpha + (j + 1) * nv);
    g.e.assign(N, 0);
    if (eps) for (int k = 0; k < N; ++k) g.e[k] = eps[j * N + k];
    else g.e[j] = 1;
    t0.G.push_back(g);
  }
  std::vector<Term> cur{t0}, nxt;
  for (int s = 0; s < m; ++s) {
    int p = order ? order[s] : s;
    if (p < 0 || p >= m) return fail("bad integration order");
    if (sum_variable(cur, p, vb[p] != 0, vb, nxt) != 0) return -1;
    cur.swap(nxt);
  }
  S.terms = cur;
  return 0;
}

// ---------------------------------------------------------------------------------------
// Fermi/Bose factors and their derivatives.
// g = g_sigma(x) and h = 1 - g obey dg/dx = -beta g h and dh/dx = +beta g h for both
// sigma, so d^k g/dx^k is a homogeneous polynomial of degree k+1 in (g, h).  g and h are
// formed from y = exp(-beta |x|) (exact in relative terms for the tails, where g or h is
// tiny) and, for sigma = -1, 1 - y = -expm1(-beta |x|) (exact in relative terms near x = 0).
// ---------------------------------------------------------------------------------------
struct GH { double g, h; };

GH fermi_gh(int sigma, double beta, double x) {
  double nt = -beta * std::fabs(x);
  double y = std::exp(nt);
  double D = sigma == 1 ? 1.0 + y : -std::expm1(nt);   // 1 + sigma y
  double sy = sigma * y;
  if (x <= 0) return {1.0 / D, sy / D};
  return {sy / D, 1.0 / D};
}

// coefficients of g^i h^(k+1-i), i = 0..k+1, of the k-th derivative (powers of beta apart)
std::vector<double> deriv_poly(int k) {
  std::vector<double> c = {0.0, 1.0};               // k = 0: g  (index = power of g)
  for (int d = 0; d < k; ++d) {
    int deg = d + 1;                                 // current total degree
    std::vector<double> n(deg + 2, 0.0);
    for (int i = 0; i <= deg; ++i) {
      int j = deg - i;                               // power of h
      if (c[i] == 0.0) continue;
      // d(g^i h^j) = -i g^i h^(j+1) + j g^(i+1) h^j   (times beta)
      n[i] += -i * c[i];
      n[i + 1] += j * c[i];
    }
    c.swap(n);
  }
  return c;
}

double fermi_deriv(int sigma, int k, double beta, double x, double* env) {
  GH v = fermi_gh(sigma, beta, x);
  std::vector<double> c = deriv_poly(k);
  double s = 0.0, a = 0.0;
  for (int i = 0; i <= k + 1; ++i) {
    double mono = std::pow(v.g, i) * std::pow(v.h, k + 1 - i);
    s += c[i] * mono;
    a += std::fabs(c[i] * mono);
  }
  double bk = std::pow(beta, k);
  if (env) *env = bk * a;
  return bk * s;
}

// c.E with an fma chain in index order
double combo(const std::vector<int>& c, const double* E) {
  double x = 0.0;
  for (size_t j = 0; j < c.size(); ++j)
    if (c[j] != 0) x = std::fma((double)c[j], E[j], x);
  return x;
}

// D = sum_q a_{m+q} X_q + e.E for the external frequencies X_0..X_{n_ext-1} of one frequency row
// (the internal ones are summed away; X = i nu_ext or its continuation omega + i Gamma).
cplx den_value(const GFac& g, const double* E, const cplx* X, int nv, int n_ext) {
  const int m = nv - n_ext;
  double re = combo(g.e, E), im = 0.0;
  for (int q = 0; q < n_ext; ++q) {
    double a = g.a[m + q];
    re = std::fma(a, X[q].real(), re);
    im += a * X[q].imag();
  }
  return cplx(re, im);
}

struct Neumaier {
  double s = 0.0, c = 0.0;
  void add(double v) {
    double t = s + v;
    if (std::fabs(s) >= std::fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
  }
  double value() const { return s + c; }
};

// sum_j |c_j|: how far c.E can move when every base energy moves by at most one unit
double l1(const std::vector<int>& c) {
  double a = 0.0;
  for (int v : c) a += std::fabs((double)v);
  return a;
}

// One sample, one frequency: value, sum |term|, the rounding envelope
// sum_t |A| prod env(F) prod |G|, and the sensitivity to the base energies
// sum_t sum_j |d term_t / d E_j|, bounded factor by factor with the product rule on magnitudes:
// a factor v(x) of argument x = c.E contributes |v'(x)| sum_j |c_j| times the other factors'
// magnitudes (v' = g^(k+1) for a Fermi/Bose factor, -1/D^2 for a Green's function).
void eval_one(const Solution& S, const double* E, const cplx* X, double beta, cplx* val, double* abs_sum,
              double* envelope, double* sens = nullptr) {
  Neumaier re, im;
  double as = 0.0, en = 0.0, se = 0.0;
  for (const Term& T : S.terms) {
    double ft = T.A, ft_env = std::fabs(T.A);
    double mag = std::fabs(S.prefactor * T.A), sm = 0.0;   // running |product| and its sensitivity
    for (const FFac& f : T.F) {
      double e;
      double x = combo(f.c, E);
      double v = fermi_deriv(f.sigma, f.k, beta, x, &e);
      ft *= v;
      ft_env *= e;
      if (sens) {
        double dv = std::fabs(fermi_deriv(f.sigma, f.k + 1, beta, x, nullptr)) * l1(f.c);
        sm = sm * std::fabs(v) + mag * dv;
        mag *= std::fabs(v);
      }
    }
    cplx r = 1.0;
    for (const GFac& g : T.G) {
      cplx rg = 1.0 / den_value(g, E, X, S.nv, S.n_ext);
      r *= rg;
      if (sens) {
        double a = std::abs(rg);
        sm = sm * a + mag * a * a * l1(g.e);
        mag *= a;
      }
    }
    cplx term = S.prefactor * ft * r;
    re.add(term.real());
    im.add(term.imag());
    as += std::abs(term);
    en += std::fabs(S.prefactor) * ft_env * std::abs(r);
    se += sm;
  }
  *val = cplx(re.value(), im.value());
  if (abs_sum) *abs_sum = as;
  if (envelope) *envelope = en;
  if (sens) *sens = se;
}

// Forward-mode dual numbers: value and derivative along one seeded direction.
struct Dual {
  cplx v, d;
};
Dual dmul(Dual a, Dual b) { return {a.v * b.v, a.d * b.v + a.v * b.d}; }

// X, dX: the n_ext external frequencies of the row and their directions.
// der_env: the rounding envelope of the derivative (the product rule applied to magnitudes).
// sens: sum_t sum_j |d term_t / d E_j| (as in eval_one); dsens: sum_t sum_j |d (d term_t) / d E_j|,
// the sensitivity of the derivative to the base energies, from the second-order product rule on
// magnitudes: with a = |v|, b = |v' dx|, s = |v'| sum|c|, q = |v'' dx| sum|c| per factor,
// (V, D, S, Q) <- (V a, D a + V b, S a + V s, Q a + D s + S b + V q).
void eval_one_dual(const Solution& S, const double* E, const double* dE, const cplx* X, const cplx* dX,
                   double beta, cplx* val, cplx* der, double* der_env, double* sens = nullptr,
                   double* dsens = nullptr) {
  const int m = S.nv - S.n_ext;
  Neumaier vr, vi, dr, di;
  double env = 0.0, se = 0.0, dse = 0.0;
  for (const Term& T : S.terms) {
    Dual t{cplx(S.prefactor * T.A), 0.0};
    // rounding envelope of the derivative: the same product rule on magnitudes
    double ev = std::fabs(S.prefactor * T.A), ed = 0.0;
    double MV = ev, MD = 0.0, MS = 0.0, MQ = 0.0;
    for (const FFac& f : T.F) {
      double x = combo(f.c, E);
      double dx = 0.0, adx = 0.0;
      for (size_t j = 0; j < f.c.size(); ++j) { dx += f.c[j] * dE[j]; adx += std::fabs(f.c[j] * dE[j]); }
      double e0, e1;
      double p = fermi_deriv(f.sigma, f.k, beta, x, &e0);
      double p1 = fermi_deriv(f.sigma, f.k + 1, beta, x, &e1);
      double dp = p1 * dx;
      t = dmul(t, Dual{cplx(p), cplx(dp)});
      ed = ed * e0 + ev * e1 * adx;
      ev = ev * e0;
      if (sens || dsens) {
        double p2 = fermi_deriv(f.sigma, f.k + 2, beta, x, nullptr);
        double a = std::fabs(p), b = std::fabs(p1) * adx, s1 = std::fabs(p1) * l1(f.c);
        double q = std::fabs(p2) * adx * l1(f.c);
        MQ = MQ * a + MD * s1 + MS * b + MV * q;
        MS = MS * a + MV * s1;
        MD = MD * a + MV * b;
        MV = MV * a;
      }
    }
    for (const GFac& g : T.G) {
      cplx D = den_value(g, E, X, S.nv, S.n_ext);
      double dEe = 0.0, adEe = 0.0;
      for (size_t j = 0; j < g.e.size(); ++j) { dEe += g.e[j] * dE[j]; adEe += std::fabs(g.e[j] * dE[j]); }
      cplx dD = dEe;
      double adX = 0.0;
      for (int q = 0; q < S.n_ext; ++q) {
        double a = (double)g.a[m + q];
        dD += a * dX[q];
        adX += std::fabs(a) * std::abs(dX[q]);
      }
      cplx r = 1.0 / D;
      t = dmul(t, Dual{r, -dD * r * r});
      double ar = std::abs(r);
      ed = ed * ar + ev * (adEe + adX) * ar * ar;
      ev = ev * ar;
      if (sens || dsens) {
        double a = ar, b = (adEe + adX) * ar * ar, s1 = ar * ar * l1(g.e);
        double q = 2.0 * ar * ar * ar * (adEe + adX) * l1(g.e);
        MQ = MQ * a + MD * s1 + MS * b + MV * q;
        MS = MS * a + MV * s1;
        MD = MD * a + MV * b;
        MV = MV * a;
      }
    }
    vr.add(t.v.real()); vi.add(t.v.imag());
    dr.add(t.d.real()); di.add(t.d.imag());
    env += ed;
    se += MS;
    dse += MQ;
  }
  *val = cplx(vr.value(), vi.value());
  *der = cplx(dr.value(), di.value());
  if (der_env) *der_env = env;
  if (sens) *sens = se;
  if (dsens) *dsens = dse;
}

// Lattice parameters (t, t', mu, k_ext) and the per-line momenta of one sample.
struct Lattice { double t, tp, mu, kx, ky; };

void line_momenta(int N, int nv, const int* alpha, const double* kx_int, const double* ky_int,
                  const Lattice& L, double* Kx, double* Ky) {
  for (int j = 0; j < N; ++j) {
    double ax = 0.0, ay = 0.0;
    for (int l = 0; l < nv; ++l) {
      int c = alpha[j * nv + l];
      if (c == 0) continue;
      double qx = l == nv - 1 ? L.kx : kx_int[l];
      double qy = l == nv - 1 ? L.ky : ky_int[l];
      ax = std::fma((double)c, qx, ax);
      ay = std::fma((double)c, qy, ay);
    }
    Kx[j] = ax;
    Ky[j] = ay;
  }
}

void sample_energies(int N, int nv, const int* alpha, const Lattice& L, uint64_t seed, uint64_t s,
                     double* E, double* Kx, double* Ky) {
  int m = nv - 1;
  std::vector<double> kx(m), ky(m);
  for (int l = 0; l < m; ++l) sample_momentum(seed, s, l, &kx[l], &ky[l]);
  line_momenta(N, nv, alpha, kx.data(), ky.data(), L, Kx, Ky);
  for (int j = 0; j < N; ++j) E[j] = line_energy(Kx[j], Ky[j], L.t, L.tp, L.mu);
}

// ---------------------------------------------------------------------------------------
// Brute-force truncated Matsubara sum of the starting integrand (Eq. goal) over the m = nv - n_ext
// internal variables, the n_ext external frequencies held fixed:
// beta^-m sum over |n_l| window of prod_j 1/(X_j + E_j).  Fermionic nu = (2n+1) pi / beta for
// n in [-nmax, nmax-1]; bosonic nu = 2 n pi / beta for n in [-nmax, nmax].
// ---------------------------------------------------------------------------------------
cplx brute_force(int N, int nv, int n_ext, const int* alpha, const int* eps, const int* boson, const double* E,
                 const cplx* X, double beta, int nmax) {
  int m = nv - n_ext;
  std::vector<double> lineE(N, 0.0);
  for (int j = 0; j < N; ++j) {
    if (eps) { for (int k = 0; k < N; ++k) lineE[j] += eps[j * N + k] * E[k]; }
    else lineE[j] = E[j];
  }
  std::vector<int> lo(m), hi(m), n(m);
  for (int l = 0; l < m; ++l) {
    bool b = boson && boson[l];
    lo[l] = -nmax;
    hi[l] = b ? nmax : nmax - 1;
    n[l] = lo[l];
  }
  const double pi = 3.141592653589793;
  Neumaier re, im;
  while (true) {
    cplx prod = 1.0;
    for (int j = 0; j < N; ++j) {
      double w = 0.0;
      for (int l = 0; l < m; ++l) {
        int c = alpha[j * nv + l];
        if (!c) continue;
        bool b = boson && boson[l];
        w += c * (b ? 2.0 * n[l] * pi / beta : (2.0 * n[l] + 1.0) * pi / beta);
      }
      cplx xj = cplx(0.0, w);
      for (int q = 0; q < n_ext; ++q) xj += (double)alpha[j * nv + m + q] * X[q];
      prod /= (xj + lineE[j]);
    }
    re.add(prod.real());
    im.add(prod.imag());
    int l = 0;
    while (l < m && ++n[l] > hi[l]) { n[l] = lo[l]; ++l; }
    if (l == m) break;
  }
  return cplx(re.value(), im.value()) / std::pow(beta, m);
}

// ---------------------------------------------------------------------------------------
// Hubbard self-energy diagrams by brute-force Wick contraction.
// Interaction line i (0..m-1) has an up vertex and a down vertex (U n_up n_down).  An up
// permutation pu over m+1 slots (slot m = external: pu[m] is where the incoming leg
// enters, the up vertex v with pu[v] == m emits the outgoing leg) and a down permutation pd
// over m slots are one contraction.  Kept: connected, one-particle irreducible, no
// single-line loops and no tadpoles (an interaction line carrying zero momentum).  Weight
// (-U)^m (-1)^F with F closed loops; the m! relabellings of interaction lines are removed by
// canonical relabelling (automorphisms are trivial once the external legs are fixed).
// Canonical relabelling: follow the up chain from the incoming leg, numbering interaction
// lines on first visit; then for each numbered line in order, walk the closed up cycle
// through its up vertex (if not yet walked) and then the down cycle through its down vertex,
// numbering new lines on first visit.
// Lines of the labelled diagram: up lines by source (skipping the outgoing leg), then down
// lines by source.  Momenta: a BFS spanning tree from the line where the external leg enters
// (lines scanned in index order); each non-tree line carries its own loop variable, in line
// order; the external momentum runs along the tree path from entry to exit.  Lines with
// equal momentum labels share one base energy.
// ---------------------------------------------------------------------------------------
struct Diagram {
  std::vector<int> code;      // canonical (pu[ext], pu[0], pd[0], pu[1], pd[1], ...)
  std::vector<int> alpha;     // [N][m+1]
  std::vector<int> eps;       // [N][N]
  double sign = 1.0;          // (-1)^F
  int loops = 0;
};

bool canonical(int m, const std::vector<int>& pu, const std::vector<int>& pd, std::vector<int>& code) {
  std::vector<int> lab(m, -1), order;
  auto visit = [&](int node) { if (lab[node] < 0) { lab[node] = (int)order.size(); order.push_back(node); } };
  std::vector<char> up_done(m, 0), dn_done(m, 0);
  for (int v = pu[m]; v != m; v = pu[v]) { visit(v); up_done[v] = 1; }
  for (size_t idx = 0; idx < order.size(); ++idx) {
    int i = order[idx];
    if (!up_done[i]) { int v = i; do { visit(v); up_done[v] = 1; v = pu[v]; } while (v != i); }
    if (!dn_done[i]) { int v = i; do { visit(v); dn_done[v] = 1; v = pd[v]; } while (v != i); }
  }
  if ((int)order.size() != m) return false;   // disconnected
  code.assign(1 + 2 * m, 0);
  auto L = [&](int v) { return v == m ? m : lab[v]; };
  code[0] = L(pu[m]);
  for (int c = 0; c < m; ++c) {
    int i = order[c];
    code[1 + 2 * c] = L(pu[i]);
    code[2 + 2 * c] = L(pd[i]);
  }
  return true;
}

// label a canonical diagram; returns false if reducible or a tadpole
bool label(int m, const std::vector<int>& code, Diagram& d) {
  int N = 2 * m - 1, nv = m + 1;
  std::vector<int> pu(m + 1), pd(m);
  pu[m] = code[0];
  for (int c = 0; c < m; ++c) { pu[c] = code[1 + 2 * c]; pd[c] = code[2 + 2 * c]; }
  struct Line { int src, dst; };
  std::vector<Line> lines;
  int exit_node = -1;
  for (int c = 0; c < m; ++c) {
    if (pu[c] == m) { exit_node = c; continue; }
    lines.push_back({c, pu[c]});
  }
  for (int c = 0; c < m; ++c) lines.push_back({c, pd[c]});
  if ((int)lines.size() != N || exit_node < 0) return false;
  int entry = pu[m];
  // BFS spanning tree
  std::vector<char> seen(m, 0), tree(N, 0);
  std::vector<int> parent_line(m, -1), queue{entry};
  seen[entry] = 1;
  for (size_t qi = 0; qi < queue.size(); ++qi) {
    int u = queue[qi];
    for (int j = 0; j < N; ++j) {
      int o = lines[j].src == u ? lines[j].dst : (lines[j].dst == u ? lines[j].src : -1);
      if (o < 0 || seen[o]) continue;
      seen[o] = 1; tree[j] = 1; parent_line[o] = j; queue.push_back(o);
    }
  }
  std::vector<int> alpha(N * nv, 0);
  // path from node x up to the root: adds `sgn` times the flow root->x along each tree line
  auto add_root_to = [&](int x, int var, int sgn) {
    while (x != entry) {
      int j = parent_line[x];
      int par = lines[j].src == x ? lines[j].dst : lines[j].src;
      int dir = lines[j].dst == x ? 1 : -1;   // line oriented par->x ?
      alpha[j * nv + var] += sgn * dir;
      x = par;
    }
  };
  int var = 0;
  for (int j = 0; j < N; ++j) {
    if (tree[j]) continue;
    if (var >= m) return false;
    alpha[j * nv + var] = 1;
    // loop: src -> dst along the chord, back dst -> src through the tree
    add_root_to(lines[j].dst, var, -1);
    add_root_to(lines[j].src, var, +1);
    ++var;
  }
  if (var != m) return false;
  add_root_to(exit_node, m, +1);   // external flow entry -> exit
  // one-particle irreducible: no line free of loop momenta
  for (int j = 0; j < N; ++j) {
    bool any = false;
    for (int l = 0; l < m; ++l) if (alpha[j * nv + l]) any = true;
    if (!any) return false;
  }
  // tadpole: zero transfer through an interaction line (up side: out - in)
  for (int c = 0; c < m; ++c) {
    std::vector<int> q(nv, 0);
    // up lines are lines[0 .. m-2]; the external legs stand in where none leaves or enters
    int jout = -1, jin = -1;
    for (int j = 0; j < m - 1; ++j) { if (lines[j].src == c) jout = j; if (lines[j].dst == c) jin = j; }
    for (int l = 0; l < nv; ++l) {
      int out = jout >= 0 ? alpha[jout * nv + l] : (l == m ? 1 : 0);
      int in = jin >= 0 ? alpha[jin * nv + l] : (l == m ? 1 : 0);
      q[l] = out - in;
    }
    if (std::all_of(q.begin(), q.end(), [](int v) { return v == 0; })) return false;
  }
  // equal momentum labels share a base energy
  std::vector<int> eps(N * N, 0);
  for (int j = 0; j < N; ++j) {
    int rep = j;
    for (int k = 0; k < j; ++k)
      if (std::equal(alpha.begin() + j * nv, alpha.begin() + (j + 1) * nv, alpha.begin() + k * nv)) { rep = k; break; }
    eps[j * N + rep] = 1;
  }
  // closed loops
  int F = 0;
  std::vector<char> vis(m, 0);
  for (int c = 0; c < m; ++c) {   // up cycles not through the external slot
    if (vis[c]) continue;
    bool ext = false;
    int v = c, len = 0;
    do { if (v == m) { ext = true; break; } vis[v] = 1; v = pu[v]; ++len; } while (v != c && len <= m + 1);
    if (!ext) ++F;
  }
  std::fill(vis.begin(), vis.end(), 0);
  for (int c = 0; c < m; ++c) {
    if (vis[c]) continue;
    int v = c;
    do { vis[v] = 1; v = pd[v]; } while (v != c);
    ++F;
  }
  d.code = code;
  d.alpha = alpha;
  d.eps = eps;
  d.loops = F;
  d.sign = (F % 2) ? -1.0 : 1.0;
  return true;
}

std::vector<Diagram> enumerate_sigma(int m) {
  std::vector<int> pu(m + 1), pd(m);
  for (int i = 0; i <= m; ++i) pu[i] = i;
  std::set<std::vector<int>> codes;
  do {
    if (pu[m] == m) continue;
    bool selfloop = false;
    for (int v = 0; v < m; ++v) if (pu[v] == v) selfloop = true;
    if (selfloop) continue;
    for (int i = 0; i < m; ++i) pd[i] = i;
    do {
      bool sl = false;
      for (int v = 0; v < m; ++v) if (pd[v] == v) sl = true;
      if (sl) continue;
      std::vector<int> code;
      if (!canonical(m, pu, pd, code)) continue;
      codes.insert(code);
    } while (std::next_permutation(pd.begin(), pd.end()));
  } while (std::next_permutation(pu.begin(), pu.end()));
  std::vector<Diagram> out;
  for (const auto& c : codes) {
    Diagram d;
    if (label(m, c, d)) out.push_back(d);
  }
  return out;
}

std::vector<Diagram> g_diagrams;

}  // namespace

// =======================================================================================
// C entry points (loaded with ctypes by the tests).  Every function returns 0 on success and
// a negative value on failure; orc_last_error() gives the reason.
// =======================================================================================
extern "C" {

const char* orc_last_error() { return g_err.c_str(); }

void orc_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox(ctr, key, out); }

// sin and cos as the oracle's dispersion uses them (the C library's).
void orc_sincos(const double* k, int64_t n, double* s, double* c) {
  for (int64_t i = 0; i < n; ++i) { s[i] = std::sin(k[i]); c[i] = std::cos(k[i]); }
}

double orc_fermi_deriv(int sigma, int k, double beta, double x) {
  return fermi_deriv(sigma, k, beta, x, nullptr);
}

// n_ext external variables, the last n_ext columns of alpha; the first n_vars - n_ext are summed.
void* orc_construct_ext(int n_lines, int n_vars, int n_ext, const int* alpha, const int* eps,
                        const int* var_is_boson, const int* order, double prefactor) {
  Solution* S = new Solution;
  if (construct(n_lines, n_vars, n_ext, alpha, eps, var_is_boson, order, prefactor, *S) != 0) {
    delete S;
    return nullptr;
  }
  return S;
}

void* orc_construct(int n_lines, int n_vars, const int* alpha, const int* eps, const int* var_is_boson,
                    const int* order, double prefactor) {
  return orc_construct_ext(n_lines, n_vars, 1, alpha, eps, var_is_boson, order, prefactor);
}

void orc_destroy(void* s) { delete (Solution*)s; }

// info[0] terms, [1] total Fermi factors, [2] total G factors (with powers),
// [3] max derivative order, [4] max G factors in a term, [5] distinct (c up to sign, sigma)
// Fermi arguments, [6] distinct (e, external coefficients) denominators
void orc_info(const void* sp, int64_t* info) {
  const Solution& S = *(const Solution*)sp;
  int64_t nf = 0, ng = 0, kmax = 0, gmax = 0;
  std::set<std::pair<std::vector<int>, int>> poles;
  std::set<std::vector<int>> dens;
  for (const Term& T : S.terms) {
    nf += (int64_t)T.F.size();
    ng += (int64_t)T.G.size();
    gmax = std::max<int64_t>(gmax, (int64_t)T.G.size());
    for (const FFac& f : T.F) {
      kmax = std::max<int64_t>(kmax, f.k);
      std::vector<int> c = f.c;
      for (int v : f.c) { if (v != 0) { if (v < 0) for (int& w : c) w = -w; break; } }
      poles.insert({c, f.sigma});
    }
    for (const GFac& g : T.G) {
      std::vector<int> key = g.e;
      for (int q = S.nv - S.n_ext; q < S.nv; ++q) key.push_back(g.a[q]);
      dens.insert(key);
    }
  }
  info[0] = (int64_t)S.terms.size(); info[1] = nf; info[2] = ng; info[3] = kmax; info[4] = gmax;
  info[5] = (int64_t)poles.size(); info[6] = (int64_t)dens.size();
}

// Term t: A, and the factor lists.  fc: [nF][N] energy coefficients, fs: sigma, fk: order,
// ge: [nG][N], ga: [nG][n_ext] external-frequency coefficients.  Sizes are returned in nF, nG.
int orc_term(const void* sp, int64_t t, double* A, int* nF, int* fc, int* fs, int* fk, int* nG,
             int* ge, int* ga, int cap) {
  const Solution& S = *(const Solution*)sp;
  if (t < 0 || t >= (int64_t)S.terms.size()) return fail("term index");
  const Term& T = S.terms[t];
  *A = T.A;
  *nF = (int)T.F.size();
  *nG = (int)T.G.size();
  if ((int)T.F.size() > cap || (int)T.G.size() > cap) return fail("cap");
  for (size_t i = 0; i < T.F.size(); ++i) {
    for (int j = 0; j < S.N; ++j) fc[i * S.N + j] = T.F[i].c[j];
    fs[i] = T.F[i].sigma; fk[i] = T.F[i].k;
  }
  for (size_t i = 0; i < T.G.size(); ++i) {
    for (int j = 0; j < S.N; ++j) ge[i * S.N + j] = T.G[i].e[j];
    for (int q = 0; q < S.n_ext; ++q) ga[i * S.n_ext + q] = T.G[i].a[S.nv - S.n_ext + q];
  }
  return 0;
}

// Energy input: E [n_e][N] (base energies), X [n_f][n_ext] complex (one row of external
// frequencies per f); out [n_f][n_e] complex, abs_sum and envelope [n_f][n_e] (either may be NULL).
int orc_eval_energies(const void* sp, const double* E, int64_t n_e, const double* X_re, const double* X_im,
                      int n_f, double beta, double* out_re, double* out_im, double* abs_sum,
                      double* envelope, double* sens, int n_threads) {
  const Solution& S = *(const Solution*)sp;
  auto work = [&](int64_t lo, int64_t hi) {
    std::vector<cplx> Xf(S.n_ext);
    for (int64_t i = lo; i < hi; ++i)
      for (int f = 0; f < n_f; ++f) {
        cplx v;
        double a, e, sn;
        for (int q = 0; q < S.n_ext; ++q) Xf[q] = cplx(X_re[f * S.n_ext + q], X_im[f * S.n_ext + q]);
        eval_one(S, E + i * S.N, Xf.data(), beta, &v, &a, &e, sens ? &sn : nullptr);
        int64_t o = (int64_t)f * n_e + i;
        out_re[o] = v.real(); out_im[o] = v.imag();
        if (abs_sum) abs_sum[o] = a;
        if (envelope) envelope[o] = e;
        if (sens) sens[o] = sn;
      }
  };
  if (n_threads <= 1) { work(0, n_e); return 0; }
  std::vector<std::thread> th;
  for (int k = 0; k < n_threads; ++k)
    th.emplace_back(work, n_e * k / n_threads, n_e * (k + 1) / n_threads);
  for (auto& x : th) x.join();
  return 0;
}

// Momentum sampling of the base energies (the per-line energies E_j = mu - eps(k_j)).
// lat = {t, t', mu, kx_ext, ky_ext}; E [n][N]; k_int (optional) [n][m][2].
int orc_sample_energies(int n_lines, int n_vars, const int* alpha, const double* lat, uint64_t seed,
                        uint64_t offset, int64_t n, double* E, double* k_int) {
  Lattice L{lat[0], lat[1], lat[2], lat[3], lat[4]};
  std::vector<double> Kx(n_lines), Ky(n_lines);
  int m = n_vars - 1;
  for (int64_t i = 0; i < n; ++i) {
    sample_energies(n_lines, n_vars, alpha, L, seed, offset + i, E + i * n_lines, Kx.data(), Ky.data());
    if (k_int)
      for (int l = 0; l < m; ++l)
        sample_momentum(seed, offset + i, l, &k_int[(i * m + l) * 2], &k_int[(i * m + l) * 2 + 1]);
  }
  return 0;
}

// Momentum mode: per-sample values [n_f][n] (optional), rounding envelope and energy sensitivity
// sum_t sum_j |d term_t / d E_j| [n_f][n] (each optional), and the Monte Carlo mean [n_f]
// (complex) and unbiased variances of Re and Im [n_f][2] (Sec. 2.3, "summing the rows": the
// mean over samples; the variance divides by n - 1).
// alpha is the labelling used for the momenta (rows of the construction's alpha).
int orc_eval_momenta(const void* sp, const int* alpha, const double* lat, uint64_t seed, uint64_t offset,
                     int64_t n, const double* X_re, const double* X_im, int n_f, double beta,
                     double* per_re, double* per_im, double* envelope, double* sens, double* mean,
                     double* var, int n_threads) {
  const Solution& S = *(const Solution*)sp;
  if (S.n_ext != 1) return fail("momentum sampling takes one external momentum (n_ext = 1)");
  Lattice L{lat[0], lat[1], lat[2], lat[3], lat[4]};
  std::vector<double> vr((size_t)n * n_f), vi((size_t)n * n_f);
  auto work = [&](int64_t lo, int64_t hi) {
    std::vector<double> E(S.N), Kx(S.N), Ky(S.N);
    for (int64_t i = lo; i < hi; ++i) {
      sample_energies(S.N, S.nv, alpha, L, seed, offset + i, E.data(), Kx.data(), Ky.data());
      for (int f = 0; f < n_f; ++f) {
        cplx v;
        double e, sn;
        const cplx Xf(X_re[f], X_im[f]);
        eval_one(S, E.data(), &Xf, beta, &v, nullptr, &e, sens ? &sn : nullptr);
        size_t o = (size_t)f * n + i;
        vr[o] = v.real(); vi[o] = v.imag();
        if (envelope) envelope[o] = e;
        if (sens) sens[o] = sn;
      }
    }
  };
  if (n_threads <= 1) work(0, n);
  else {
    std::vector<std::thread> th;
    for (int k = 0; k < n_threads; ++k) th.emplace_back(work, n * k / n_threads, n * (k + 1) / n_threads);
    for (auto& x : th) x.join();
  }
  for (int f = 0; f < n_f; ++f) {
    const double* r = vr.data() + (size_t)f * n;
    const double* im = vi.data() + (size_t)f * n;
    Neumaier sr, si;
    for (int64_t i = 0; i < n; ++i) { sr.add(r[i]); si.add(im[i]); }
    double mr = sr.value() / n, mi = si.value() / n;
    Neumaier qr, qi;
    for (int64_t i = 0; i < n; ++i) { qr.add((r[i] - mr) * (r[i] - mr)); qi.add((im[i] - mi) * (im[i] - mi)); }
    if (mean) { mean[2 * f] = mr; mean[2 * f + 1] = mi; }
    if (var) { var[2 * f] = n > 1 ? qr.value() / (n - 1) : 0.0; var[2 * f + 1] = n > 1 ? qi.value() / (n - 1) : 0.0; }
    if (per_re) std::memcpy(per_re + (size_t)f * n, r, sizeof(double) * n);
    if (per_im) std::memcpy(per_im + (size_t)f * n, im, sizeof(double) * n);
  }
  return 0;
}

// Dual-number derivative of the per-sample value along one direction (der_env, optional: the
// rounding envelope of the derivative, the product rule applied to magnitudes; sens and dsens,
// optional: the energy sensitivities of the value and of the derivative, as in eval_one_dual):
// which = 0: d/d omega (X -> X + h, the same shift for every frequency; the derivative of
// Sigma_f is with respect to its own omega_f), 1: d/d mu, 2: d/d kx_ext, 3: d/d ky_ext.
// der [n_f][n] complex (re, im arrays).
int orc_eval_momenta_deriv(const void* sp, const int* alpha, const double* lat, uint64_t seed,
                           uint64_t offset, int64_t n, const double* X_re, const double* X_im, int n_f,
                           double beta, int which, double* val_re, double* val_im, double* der_re,
                           double* der_im, double* der_env, double* sens, double* dsens, int n_threads) {
  const Solution& S = *(const Solution*)sp;
  if (S.n_ext != 1) return fail("momentum sampling takes one external momentum (n_ext = 1)");
  Lattice L{lat[0], lat[1], lat[2], lat[3], lat[4]};
  int nv = S.nv;
  auto work = [&](int64_t lo, int64_t hi) {
    std::vector<double> E(S.N), Kx(S.N), Ky(S.N), dE(S.N);
    for (int64_t i = lo; i < hi; ++i) {
      sample_energies(S.N, nv, alpha, L, seed, offset + i, E.data(), Kx.data(), Ky.data());
      for (int j = 0; j < S.N; ++j) {
        double aext = alpha[j * nv + nv - 1];
        if (which == 1) dE[j] = 1.0;
        else if (which == 2) dE[j] = -aext * deps_dkx(Kx[j], Ky[j], L.t, L.tp);
        else if (which == 3) dE[j] = -aext * deps_dkx(Ky[j], Kx[j], L.t, L.tp);
        else dE[j] = 0.0;
      }
      cplx dX = which == 0 ? cplx(1.0, 0.0) : cplx(0.0, 0.0);
      for (int f = 0; f < n_f; ++f) {
        cplx v, d;
        double de, sn, dsn;
        const cplx Xf(X_re[f], X_im[f]);
        eval_one_dual(S, E.data(), dE.data(), &Xf, &dX, beta, &v, &d, &de, sens ? &sn : nullptr,
                      dsens ? &dsn : nullptr);
        size_t o = (size_t)f * n + i;
        if (val_re) { val_re[o] = v.real(); val_im[o] = v.imag(); }
        der_re[o] = d.real(); der_im[o] = d.imag();
        if (der_env) der_env[o] = de;
        if (sens) sens[o] = sn;
        if (dsens) dsens[o] = dsn;
      }
    }
  };
  if (n_threads <= 1) work(0, n);
  else {
    std::vector<std::thread> th;
    for (int k = 0; k < n_threads; ++k) th.emplace_back(work, n * k / n_threads, n * (k + 1) / n_threads);
    for (auto& x : th) x.join();
  }
  return 0;
}

// Dual-number derivative with energy input: dE [n_e][N] direction for the base energies,
// X [n_f][n_ext] the frequency rows, dX [n_ext] the direction of the external frequencies
// (the same for every row).  dsens [n_f][n_e] (optional): the derivative's energy sensitivity.
int orc_eval_energies_deriv(const void* sp, const double* E, const double* dE, int64_t n_e,
                            const double* X_re, const double* X_im, const double* dX_re, const double* dX_im,
                            int n_f, double beta, double* der_re, double* der_im, double* dsens) {
  const Solution& S = *(const Solution*)sp;
  std::vector<cplx> Xf(S.n_ext), dX(S.n_ext);
  for (int q = 0; q < S.n_ext; ++q) dX[q] = cplx(dX_re[q], dX_im[q]);
  for (int64_t i = 0; i < n_e; ++i)
    for (int f = 0; f < n_f; ++f) {
      cplx v, d;
      for (int q = 0; q < S.n_ext; ++q) Xf[q] = cplx(X_re[f * S.n_ext + q], X_im[f * S.n_ext + q]);
      double dsn;
      eval_one_dual(S, E + i * S.N, dE + i * S.N, Xf.data(), dX.data(), beta, &v, &d, nullptr, nullptr,
                    dsens ? &dsn : nullptr);
      der_re[(size_t)f * n_e + i] = d.real();
      der_im[(size_t)f * n_e + i] = d.imag();
      if (dsens) dsens[(size_t)f * n_e + i] = dsn;
    }
  return 0;
}

// X [n_ext]: the external frequencies (the last n_ext variables); the others are summed.
int orc_brute_force(int n_lines, int n_vars, int n_ext, const int* alpha, const int* eps,
                    const int* var_is_boson, const double* E, const double* X_re, const double* X_im,
                    double beta, int nmax, double* out) {
  if (n_ext < 1 || n_vars < n_ext + 1) return fail("bad sizes");
  std::vector<cplx> X(n_ext);
  for (int q = 0; q < n_ext; ++q) X[q] = cplx(X_re[q], X_im[q]);
  cplx v = brute_force(n_lines, n_vars, n_ext, alpha, eps, var_is_boson, E, X.data(), beta, nmax);
  out[0] = v.real();
  out[1] = v.imag();
  return 0;
}

// Enumerate; returns the number of diagrams (kept until the next call).
int orc_enumerate_sigma(int order) {
  if (order < 1 || order > 6) return fail("order out of range");
  g_diagrams = enumerate_sigma(order);
  return (int)g_diagrams.size();
}

// Diagram i of the last enumeration: alpha [N][m+1], eps [N][N], code [1+2m], sign, loops.
int orc_diagram(int i, int* alpha, int* eps, int* code, double* sign, int* loops) {
  if (i < 0 || i >= (int)g_diagrams.size()) return fail("diagram index");
  const Diagram& d = g_diagrams[i];
  std::copy(d.alpha.begin(), d.alpha.end(), alpha);
  std::copy(d.eps.begin(), d.eps.end(), eps);
  std::copy(d.code.begin(), d.code.end(), code);
  *sign = d.sign;
  *loops = d.loops;
  return 0;
}

}  // extern "C"
