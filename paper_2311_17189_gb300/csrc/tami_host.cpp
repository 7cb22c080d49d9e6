// Host side of libtami: AMI construction (Sec. 2.2), flattening of the solution into the
// device term table, and the Hubbard self-energy enumerator with its momentum labeller
// (Sec. 2.5).  This code is cold: it runs once per diagram.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "tami_internal.h"

namespace tami {

static thread_local std::string g_last_error;
void set_error(const std::string& msg) { g_last_error = msg; }

namespace {

using Factors = std::vector<std::pair<Form, int>>;

void add_factor(Factors& G, const Form& f, int q) {
  auto it = std::lower_bound(G.begin(), G.end(), f,
                             [](const std::pair<Form, int>& p, const Form& x) { return p.first < x; });
  if (it != G.end() && it->first == f) it->second += q;
  else G.insert(it, {f, q});
}

bool is_zero(const Form& f) {
  for (int8_t v : f.e) if (v) return false;
  for (int8_t v : f.a) if (v) return false;
  return true;
}

// n! and the binomial coefficient as doubles (exact for the small arguments used here)
double fact(int n) { double r = 1.0; while (n > 1) r *= n--; return r; }
double choose(int n, int k) {
  double r = 1.0;
  for (int i = 0; i < k; ++i) r = r * (n - i) / (i + 1);
  return r;
}

struct Movable {       // a Green's function left after the pole is taken out
  Form f;              // its form with z replaced by the pole position
  int q;               // power
  int arp;             // its coefficient of the summed variable (0: constant in z)
};

// Sum over nu_p of every term: residues at the poles of the z-dependent Green's functions
// (Eq. Res_Th), multipole ones through the Leibniz rule (Eq. Res_mul).
int sum_over(const std::vector<SymTerm>& in, int p, int nv, const std::vector<uint8_t>& boson,
             std::vector<SymTerm>& out) {
  out.clear();
  for (const SymTerm& T : in) {
    std::map<Form, std::vector<int>> poles;   // pole position (a linear form) -> factors
    int degree = 0;
    for (int i = 0; i < (int)T.G.size(); ++i) {
      const Form& g = T.G[i].first;
      int ap = g.a[p];
      if (ap == 0) continue;
      if (ap != 1 && ap != -1) {
        set_error("summed variable appears with a coefficient of magnitude > 1");
        return TAMI_EUNSUPPORTED;
      }
      degree += T.G[i].second;
      // root of ap z + rest: z0 = -ap * rest
      Form z0;
      for (int j = 0; j < kMaxLines; ++j) z0.e[j] = (int8_t)(-ap * g.e[j]);
      for (int l = 0; l < nv; ++l) z0.a[l] = l == p ? 0 : (int8_t)(-ap * g.a[l]);
      poles[z0].push_back(i);
    }
    if (degree < 2) {
      set_error("a term decays slower than 1/z^2 in a summed variable");
      return TAMI_EUNSUPPORTED;
    }
    for (const auto& pole : poles) {
      const Form& z0 = pole.first;
      const std::vector<int>& mem = pole.second;
      int M = 0;
      double sgn = 1.0;
      for (int i : mem) {
        M += T.G[i].second;
        if (T.G[i].first.a[p] < 0 && (T.G[i].second & 1)) sgn = -sgn;
      }
      // weight f (fermionic nu_p) or -n_B (bosonic), reduced by the Matsubara shift's parity
      FermiFactor ff;
      ff.c = z0.e;
      int parity = 0;
      for (int l = 0; l < nv; ++l)
        if (l != p && !boson[l]) parity += std::abs((int)z0.a[l]);
      int sigma = boson[p] ? -1 : 1;
      if (parity & 1) sigma = -sigma;
      ff.sigma = (int8_t)sigma;
      bool czero = std::all_of(ff.c.begin(), ff.c.end(), [](int8_t v) { return v == 0; });
      if (czero && sigma < 0) {
        set_error("Bose factor at zero energy");
        return TAMI_EUNSUPPORTED;
      }
      std::vector<Movable> rest;
      std::vector<int> zdep;
      for (int i = 0; i < (int)T.G.size(); ++i) {
        if (std::find(mem.begin(), mem.end(), i) != mem.end()) continue;
        const Form& g = T.G[i].first;
        int arp = g.a[p];
        Movable mv{g, T.G[i].second, arp};
        for (int j = 0; j < kMaxLines; ++j) {
          int v = g.e[j] + arp * z0.e[j];
          if (v > 100 || v < -100) { set_error("energy coefficient overflow"); return TAMI_EUNSUPPORTED; }
          mv.f.e[j] = (int8_t)v;
        }
        for (int l = 0; l < nv; ++l) mv.f.a[l] = (int8_t)(g.a[l] + arp * z0.a[l]);
        mv.f.a[p] = 0;
        if (is_zero(mv.f)) { set_error("vanishing denominator after substitution"); return TAMI_EUNSUPPORTED; }
        if (arp) zdep.push_back((int)rest.size());
        rest.push_back(mv);
      }
      // distribute M-1 derivatives over the weight and the z-dependent factors
      const int n = M - 1;
      // all (k_1..k_R) with sum <= n; the weight takes k_0 = n - sum (odometer)
      std::vector<int> kz(zdep.size(), 0);
      while (true) {
        int used = 0;
        for (int v : kz) used += v;
        if (used <= n) {
          int k0 = n - used;
          SymTerm nt;
          double A = T.A * sgn / fact(k0);
          for (size_t r = 0; r < zdep.size(); ++r) {
            const Movable& mv = rest[zdep[r]];
            int kr = kz[r];
            double c = choose(mv.q + kr - 1, kr);
            if ((kr & 1) && mv.arp > 0) c = -c;   // (-1)^k a^k with a = +1
            A *= c;                                // a = -1: (-1)^k (-1)^k = 1
          }
          nt.A = A;
          nt.F = T.F;
          FermiFactor f = ff;
          f.k = (int8_t)k0;
          nt.F.push_back(f);
          for (size_t i = 0; i < rest.size(); ++i) {
            int extra = 0;
            auto it = std::find(zdep.begin(), zdep.end(), (int)i);
            if (it != zdep.end()) extra = kz[it - zdep.begin()];
            add_factor(nt.G, rest[i].f, rest[i].q + extra);
          }
          out.push_back(std::move(nt));
        }
        // advance odometer
        size_t pos = 0;
        while (pos < kz.size()) {
          if (++kz[pos] <= n) break;
          kz[pos] = 0;
          ++pos;
        }
        if (pos == kz.size()) break;
      }
    }
  }
  return TAMI_OK;
}

}  // namespace

// ------------------------------------------------------------------------------ flatten
namespace {

using Vec = std::array<int8_t, kMaxLines>;

int first_sign(const Vec& v) {
  for (int8_t x : v) if (x) return x > 0 ? 1 : -1;
  return 1;
}
Vec scaled(const Vec& v, int s) {
  Vec r;
  for (int i = 0; i < kMaxLines; ++i) r[i] = (int8_t)(s * v[i]);
  return r;
}

struct Blob {
  std::vector<unsigned char> b;
  int reserve(size_t bytes) {
    size_t off = (b.size() + 15) & ~size_t(15);
    b.resize(off + ((bytes + 15) & ~size_t(15)), 0);
    return (int)off;
  }
  template <class T> T* at(int off) { return reinterpret_cast<T*>(b.data() + off); }
};

}  // namespace

DagPrefixes dag_prefixes(const int* opsb, int n_ops, const double* leafA) {
  DagPrefixes r;
  int max_node = 0;
  for (int i = 0; i < n_ops; ++i) max_node = std::max(max_node, opsb[2 * i] & kOpbDstMask);
  r.node_value.assign(max_node + 1, -1);
  r.node_sign.assign(max_node + 1, 1);
  r.op_prefix.resize(n_ops);
  r.op_sign.resize(n_ops);
  r.op_new.resize(n_ops);
  // (parent, F, operand kind, operand: a leaf by its signed coefficient's bits, a node operand by
  // its prefix and sign) -> prefix
  std::map<std::tuple<int, int, int, long long>, int> id;
  std::vector<int> cur(max_node + 1, -1), cur_sign(max_node + 1, 1);
  for (int i = 0; i < n_ops; ++i) {
    const int x = opsb[2 * i], y = opsb[2 * i + 1];
    const int dst = x & kOpbDstMask, ref = y >> kOpbRefShift;
    const bool leaf = x & kOpbLeaf;
    const int parent = (x & kOpbFirst) ? -1 : cur[dst];
    // the op's partial sum is fma(F, operand, sp * parent prefix) = sign * fma(F, sign * operand,
    // parent prefix): sign = sp with a parent; a first step takes the operand's sign out instead
    const int sp = parent < 0 ? 1 : cur_sign[dst];
    if (leaf ? leafA[ref] == 0.0 : r.node_value[ref] < 0) {
      // an operand that is identically zero (a leaf whose terms cancelled exactly, or a node made
      // only of such) adds nothing: the partial sum stays the parent's (none: zero)
      r.op_prefix[i] = parent;
      r.op_sign[i] = (signed char)sp;
      r.op_new[i] = 0;
      cur[dst] = r.node_value[dst] = parent;
      cur_sign[dst] = r.node_sign[dst] = (signed char)sp;
      continue;
    }
    const int so = leaf ? (leafA[ref] < 0 ? -1 : 1) : r.node_sign[ref];
    const int sign = parent < 0 ? so : sp;
    const DagPrefix q{parent, y & kOpbFvMask, leaf ? 0 : 1, leaf ? ref : r.node_value[ref], leaf ? sign : sign * so};
    long long key;
    if (leaf) {
      const double c = q.osign * leafA[ref];
      std::memcpy(&key, &c, sizeof key);
    } else {
      key = 2LL * q.operand + (q.osign < 0 ? 1 : 0);
    }
    const auto ins = id.emplace(std::make_tuple(q.parent, q.fv, q.node, key), (int)r.p.size());
    if (ins.second) r.p.push_back(q);
    r.op_prefix[i] = ins.first->second;
    r.op_sign[i] = (signed char)sign;
    r.op_new[i] = ins.second;
    cur[dst] = r.node_value[dst] = ins.first->second;
    cur_sign[dst] = r.node_sign[dst] = (signed char)sign;
  }
  return r;
}

int flatten(tami_diagram* d) {
  const int N = d->N, nv = d->nv, n_ext = d->n_ext, m = nv - n_ext;
  // ---- energy combinations (sign-canonical), Fermi values, denominators
  std::map<Vec, int> combo_id;
  std::vector<Vec> combos;
  auto combo = [&](const Vec& v, int* sign) {
    int s = first_sign(v);
    Vec c = scaled(v, s);
    *sign = s;
    auto it = combo_id.find(c);
    if (it != combo_id.end()) return it->second;
    int id = (int)combos.size();
    combo_id[c] = id;
    combos.push_back(c);
    return id;
  };
  struct FvKey { int u, sigma, sign, k; bool operator<(const FvKey& o) const {
      return std::tie(u, sigma, sign, k) < std::tie(o.u, o.sigma, o.sign, o.k); } };
  std::map<FvKey, int> fv_tmp;   // provisional ids, renumbered by base below
  // A complex denominator D = sum_q a_q X_q + s * (combination u).E; its external coefficients
  // are g * v_k with v_k one of the table's vectors: for one external v_0 = (1) and g = a_0, for
  // several g = 1 and v_k = a.
  struct CdKey { int u, sign, a, xk; bool operator<(const CdKey& o) const {
      return std::tie(u, sign, a, xk) < std::tie(o.u, o.sign, o.a, o.xk); } };
  using ExtVec = std::array<int8_t, kMaxExt>;
  std::map<ExtVec, int> xvec_id;
  std::vector<ExtVec> xvecs;
  if (n_ext == 1) { ExtVec one{}; one[0] = 1; xvec_id[one] = 0; xvecs.push_back(one); }
  std::map<int, int> rden_id;
  std::vector<int> rdens;
  std::map<CdKey, int> cden_id;
  std::vector<CdKey> cdens;
  struct FlatTerm {
    double A;
    std::vector<FvKey> fv;
    std::vector<std::pair<int, int>> rd, cd;   // (id, power), sorted
  };
  std::vector<FlatTerm> ft;
  ft.reserve(d->terms.size());
  int64_t nF = 0, nG = 0;
  int max_der = 0, max_g = 0;
  std::set<std::pair<Vec, int>> upoles;
  std::set<std::pair<Vec, ExtVec>> udens;
  for (const SymTerm& T : d->terms) {
    FlatTerm t;
    t.A = T.A * d->prefactor;
    for (const FermiFactor& f : T.F) {
      int s;
      int u = combo(f.c, &s);
      FvKey key{u, f.sigma, s, f.k};
      fv_tmp.emplace(key, 0);
      t.fv.push_back(key);
      max_der = std::max(max_der, (int)f.k);
      upoles.insert({combos[u], f.sigma});
      ++nF;
    }
    int gcount = 0;
    for (const auto& gq : T.G) {
      const Form& g = gq.first;
      int q = gq.second;
      gcount += q;
      nG += q;
      ExtVec av{};
      int a_first = 0;
      for (int q2 = 0; q2 < n_ext; ++q2) {
        av[q2] = g.a[m + q2];
        if (!a_first) a_first = av[q2];
      }
      Vec e = g.e;
      udens.insert({e, av});
      // canonical sign: first external coefficient > 0, else first energy coefficient > 0
      int dsign = a_first ? (a_first > 0 ? 1 : -1) : first_sign(e);
      if (dsign < 0 && (q & 1)) t.A = -t.A;     // 1/(-D)^q = (-1)^q / D^q
      e = scaled(e, dsign);
      for (int q2 = 0; q2 < n_ext; ++q2) av[q2] = (int8_t)(dsign * av[q2]);
      int s;
      int u = combo(e, &s);
      if (a_first == 0) {
        auto it = rden_id.find(u);
        int id;
        if (it == rden_id.end()) { id = (int)rdens.size(); rden_id[u] = id; rdens.push_back(u); }
        else id = it->second;
        t.rd.push_back({id, q});
      } else {
        int a = 1, xk = 0;
        if (n_ext == 1) a = av[0];
        else {
          auto xi = xvec_id.find(av);
          if (xi == xvec_id.end()) { xk = (int)xvecs.size(); xvec_id[av] = xk; xvecs.push_back(av); }
          else xk = xi->second;
        }
        CdKey key{u, s, a, xk};
        auto it = cden_id.find(key);
        int id;
        if (it == cden_id.end()) { id = (int)cdens.size(); cden_id[key] = id; cdens.push_back(key); }
        else id = it->second;
        t.cd.push_back({id, q});
      }
    }
    max_g = std::max(max_g, gcount);
    std::sort(t.rd.begin(), t.rd.end());
    std::sort(t.cd.begin(), t.cd.end());
    ft.push_back(std::move(t));
  }
  if (max_der > kMaxDer) { set_error("derivative order above the kernels' limit"); return TAMI_EUNSUPPORTED; }
  // Fermi segments: one per (combination, sigma), the Bose-type ones (sigma = -1, which need
  // 1 - e^{-beta|x|}) first; inside a segment the values by derivative order (k = 0 first), then
  // sign.  The kernels then run plain loops over segments and values, with no data-dependent
  // branches around FP64 work.
  struct Seg { int combo, sigma, v0, vk1, v1; };
  std::map<std::pair<int, int>, std::vector<FvKey>> by_seg;
  for (auto& kv : fv_tmp) by_seg[{kv.first.sigma < 0 ? 0 : 1, kv.first.u}].push_back(kv.first);
  std::vector<Seg> segs;
  std::vector<FvKey> fvs;
  int n_bose_seg = 0;
  for (auto& kv : by_seg) {
    std::vector<FvKey> list = kv.second;
    std::sort(list.begin(), list.end(), [](const FvKey& a, const FvKey& b) {
      return a.k != b.k ? a.k < b.k : a.sign < b.sign; });
    Seg g{kv.first.second, list[0].sigma, (int)fvs.size(), -1, 0};
    for (auto& k : list) {
      if (k.k >= 1 && g.vk1 < 0) g.vk1 = (int)fvs.size();
      fv_tmp[k] = (int)fvs.size();
      fvs.push_back(k);
    }
    g.v1 = (int)fvs.size();
    if (g.vk1 < 0) g.vk1 = g.v1;
    if (g.sigma < 0) ++n_bose_seg;
    segs.push_back(g);
  }
  // ---- groups: by (complex signature) and within it by (real signature)
  std::map<std::vector<std::pair<int, int>>, int> g2_id;
  std::vector<std::vector<std::pair<int, int>>> g2s;
  std::map<std::pair<std::vector<std::pair<int, int>>, std::vector<std::pair<int, int>>>, std::vector<int>> g1map;
  for (size_t i = 0; i < ft.size(); ++i) {
    if (!g2_id.count(ft[i].cd)) { g2_id[ft[i].cd] = (int)g2s.size(); g2s.push_back(ft[i].cd); }
    g1map[{ft[i].cd, ft[i].rd}].push_back((int)i);
  }
  // the group without frequency-dependent factors (if any) goes first: the kernels add its weight
  // without a product
  int g2_const = 0;
  for (size_t g = 0; g < g2s.size(); ++g)
    if (g2s[g].empty()) {
      if (g != 0) {
        std::swap(g2s[0], g2s[g]);
        for (auto& kv : g2_id) {
          if (kv.second == 0) kv.second = (int)g;
          else if (kv.second == (int)g) kv.second = 0;
        }
      }
      g2_const = 1;
      break;
    }
  struct G1 { int g2; std::vector<std::pair<int, int>> rd; std::vector<int> terms; };
  std::vector<G1> g1s;
  for (auto& kv : g1map) g1s.push_back({g2_id[kv.first.first], kv.first.second, kv.second});
  std::stable_sort(g1s.begin(), g1s.end(), [](const G1& x, const G1& y) { return x.g2 < y.g2; });

  // ---- phase-2 products: a trie over each frequency-dependent group's factors (the denominators
  // used by more groups first, each repeated by its power), so that groups sharing a leading
  // sub-product compute it once.  Values: index c < n_cden is 1/D_c itself; index n_cden + k is
  // product node k = value[src_k] * value[c_k]; each group reads the value at the end of its path.
  const int n_cd = (int)cdens.size();
  std::vector<int> cuse(n_cd, 0);
  for (auto& g : g2s) for (auto& pr : g) ++cuse[pr.first];
  std::vector<std::pair<int, int>> pnodes;   // (src value index, c)
  std::vector<int> g2node(g2s.size(), -1);
  {
    std::map<std::pair<int, int>, int> child;
    for (size_t g = 0; g < g2s.size(); ++g) {
      if (g2s[g].empty()) continue;
      auto fs = g2s[g];
      std::stable_sort(fs.begin(), fs.end(), [&](const std::pair<int, int>& a, const std::pair<int, int>& b) {
        return cuse[a.first] != cuse[b.first] ? cuse[a.first] > cuse[b.first] : a.first < b.first; });
      std::vector<int> seq;
      for (auto& pr : fs) for (int k = 0; k < pr.second; ++k) seq.push_back(pr.first);
      int cur = seq[0];
      for (size_t i = 1; i < seq.size(); ++i) {
        const auto key = std::make_pair(cur, seq[i]);
        const auto it = child.find(key);
        if (it != child.end()) { cur = it->second; continue; }
        const int v = n_cd + (int)pnodes.size();
        pnodes.push_back(key);
        child[key] = v;
        cur = v;
      }
      g2node[g] = cur;
    }
  }
  if ((int)pnodes.size() > kMaxProdNodes || (int)combos.size() > kMaxCombos || (int)fvs.size() > kMaxFermiValues ||
      (int)rdens.size() > kMaxRealDens || (int)cdens.size() > kMaxCplxDens) {
    set_error("term table exceeds the kernels' per-sample capacities: " + std::to_string(combos.size()) +
              " energy combinations (at most " + std::to_string(kMaxCombos) + "), " + std::to_string(fvs.size()) +
              " Fermi values (" + std::to_string(kMaxFermiValues) + "), " + std::to_string(rdens.size()) +
              " real denominators (" + std::to_string(kMaxRealDens) + "), " + std::to_string(cdens.size()) +
              " complex denominators (" + std::to_string(kMaxCplxDens) + "), " + std::to_string(pnodes.size()) +
              " product nodes (" + std::to_string(kMaxProdNodes) + ")");
    return TAMI_EUNSUPPORTED;
  }
  // ---- momentum labels: representative lines
  std::vector<int> repl;
  for (int j = 0; j < N; ++j) {
    bool dup = false;
    for (int k = 0; k < j; ++k)
      if (std::equal(d->alpha.begin() + j * nv, d->alpha.begin() + (j + 1) * nv, d->alpha.begin() + k * nv)) dup = true;
    if (!dup) repl.push_back(j);
  }
  // every base energy that the table reads must be computed
  std::vector<char> needed(N, 0);
  for (const Vec& c : combos) for (int j = 0; j < N; ++j) if (c[j]) needed[j] = 1;
  for (int j = 0; j < N; ++j)
    if (needed[j] && std::find(repl.begin(), repl.end(), j) == repl.end()) repl.push_back(j);
  std::sort(repl.begin(), repl.end());
  // lines carrying k_ext first: only their energies depend on k_ext (the adjoint needs sin there)
  const int n_rep_ext = (int)(std::stable_partition(repl.begin(), repl.end(), [&](int j) {
                                for (int l = m; l < nv; ++l) if (d->alpha[j * nv + l]) return true;
                                return false; }) - repl.begin());

  // ---- blob
  TableHeader& h = d->hdr;
  h = TableHeader{};
  h.N = N; h.nv = nv; h.m = m;
  h.n_ext = n_ext;
  if (xvecs.empty()) { ExtVec e0{}; e0[0] = 1; xvecs.push_back(e0); }   // no complex denominator
  h.n_xk = (int)xvecs.size();
  h.n_rep = (int)repl.size();
  h.n_rep_ext = n_rep_ext;
  h.n_combo = (int)combos.size();
  int nnz = 0;
  for (const Vec& c : combos) for (int j = 0; j < N; ++j) if (c[j]) ++nnz;
  h.combo_nnz = nnz;
  h.n_fseg = (int)segs.size();
  h.n_fseg_bose = n_bose_seg;
  h.n_fv = (int)fvs.size();
  h.n_rden = (int)rdens.size();
  h.n_cden = (int)cdens.size();
  h.n_g1 = (int)g1s.size();
  // Pole tree (Sec. 2.1, the factorised FT): per group, a tree over each term's Fermi values,
  // one level per residue step; terms with equal paths merge their coefficients at a leaf.  The
  // level a node branches on is chosen per node: the one with the fewest distinct Fermi values
  // among the node's terms (the usual greedy ordering for small decision trees; ties go to the
  // later residue step), unless the fixed reverse residue order gives fewer edges for the group.
  // Identical sub-sums are then shared (a DAG), and the group is emitted in post order as a
  // program of one fma per edge over value slots:
  //   v[dst] = F_c * (c is a leaf ? A_c : v[c]) + (c is dst's first child ? 0 : v[dst]).
  // Two encodings of the same ops: `ops` for the forward with slots reused by liveness (kOp*),
  // `opsb` for the adjoint with one slot per node, every value kept for the reverse walk (kOpb*).
  std::vector<std::pair<int, int>> ops, opsb;
  std::vector<double> leafA;
  std::vector<std::pair<int, int>> g1_ops(g1s.size());
  std::vector<int> g1_node(g1s.size() + 1, 0);
  int n_inner = 0, max_slots = 0, node_base = 0;
  const int m_depth = m;
  struct Node { int fv; std::vector<int> kids; double A; };
  auto build_tree = [&](const std::vector<int>& terms, bool greedy) {
    std::vector<Node> nodes(1, Node{-1, {}, 0.0});
    std::function<void(int, const std::vector<int>&, unsigned)> grow = [&](int u, const std::vector<int>& ts,
                                                                           unsigned left) {
      if (!left) {
        for (int ti : ts) nodes[u].A += ft[ti].A;
        return;
      }
      int best = -1;
      size_t best_n = 0;
      for (int L = m_depth - 1; L >= 0; --L) {
        if (!(left >> L & 1u)) continue;
        if (!greedy) { best = L; break; }
        std::set<int> vals;
        for (int ti : ts) vals.insert(fv_tmp[ft[ti].fv[L]]);
        if (best < 0 || vals.size() < best_n) { best = L; best_n = vals.size(); }
      }
      std::vector<int> first_seen;
      std::map<int, std::vector<int>> parts;
      for (int ti : ts) {
        const int f = fv_tmp[ft[ti].fv[best]];
        if (!parts.count(f)) first_seen.push_back(f);
        parts[f].push_back(ti);
      }
      for (int f : first_seen) {
        const int c = (int)nodes.size();
        nodes.push_back(Node{f, {}, 0.0});
        nodes[u].kids.push_back(c);
        grow(c, parts[f], left & ~(1u << best));
      }
    };
    grow(0, terms, (1u << m_depth) - 1u);
    return nodes;
  };
  for (size_t g = 0; g < g1s.size(); ++g) {
    for (int ti : g1s[g].terms)
      if ((int)ft[ti].fv.size() != m_depth) { set_error("term with an unexpected number of Fermi factors"); return TAMI_EUNSUPPORTED; }
    std::vector<Node> nodes = build_tree(g1s[g].terms, true);
    std::vector<Node> fixed = build_tree(g1s[g].terms, false);
    if (fixed.size() <= nodes.size()) nodes.swap(fixed);
    const int begin = (int)ops.size();
    // Identical sub-sums are computed once: nodes are hash-consed bottom-up on their sorted
    // (Fermi value, child) lists (a leaf is its coefficient), which turns the tree into a DAG.
    std::map<long long, int> leaf_uid;                  // coefficient bits -> index into leafA
    std::map<std::vector<std::pair<int, int>>, int> inner_uid;
    std::vector<std::vector<std::pair<int, int>>> ukids;   // (fv, child: >= 0 inner uid, < 0 -(leaf index + 1))
    std::function<int(int)> canon = [&](int u) -> int {
      if (nodes[u].kids.empty()) {
        long long bits;
        std::memcpy(&bits, &nodes[u].A, sizeof bits);
        auto it = leaf_uid.find(bits);
        if (it == leaf_uid.end()) {
          it = leaf_uid.emplace(bits, (int)leafA.size()).first;
          leafA.push_back(nodes[u].A);
        }
        return -(it->second + 1);
      }
      std::vector<std::pair<int, int>> key;
      for (int c : nodes[u].kids) key.push_back({nodes[c].fv, canon(c)});
      std::sort(key.begin(), key.end());
      auto it = inner_uid.find(key);
      if (it != inner_uid.end()) return it->second;
      const int id = (int)ukids.size();
      inner_uid.emplace(key, id);
      ukids.push_back(key);
      return id;
    };
    const int root = canon(0);
    // post order over the unique nodes, children first; node ids for the adjoint: root first
    struct Op { int dst, ref, fv, first, leaf, run; };
    std::vector<Op> gops;
    std::vector<int> gid(ukids.size(), -1);
    int n_gid = 0;
    gid[root] = n_gid++;
    std::vector<char> done(ukids.size(), 0);
    std::function<void(int)> emit = [&](int id) {
      for (auto& kr : ukids[id]) if (kr.second >= 0 && !done[kr.second]) emit(kr.second);
      if (gid[id] < 0) gid[id] = n_gid++;
      const int nk = (int)ukids[id].size();
      for (int i = 0; i < nk; ++i) {
        const auto& kr = ukids[id][i];
        const bool leaf = kr.second < 0;
        gops.push_back({id, leaf ? -kr.second - 1 : kr.second, kr.first, i == 0 ? 1 : 0, leaf ? 1 : 0,
                        leaf && i == nk - 1 ? nk : 0});
      }
      done[id] = 1;
    };
    emit(root);
    // forward slots: linear scan, a node's slot from its first edge to its last use
    std::vector<int> last_use(ukids.size(), -1), slot(ukids.size(), -1), free_slots;
    for (size_t p = 0; p < gops.size(); ++p) if (!gops[p].leaf) last_use[gops[p].ref] = (int)p;
    int n_live = 0;
    const int base = node_base;
    for (size_t p = 0; p < gops.size(); ++p) {
      const Op& o = gops[p];
      if (slot[o.dst] < 0) {
        if (!free_slots.empty()) { slot[o.dst] = free_slots.back(); free_slots.pop_back(); }
        else slot[o.dst] = n_live++;
      }
      const int fref = o.leaf ? o.ref : slot[o.ref];
      const int bref = o.leaf ? o.ref : base + gid[o.ref];
      if (o.run > 255 || n_live > kMaxSlots || base + n_gid > (1 << kOpbDstBits) || fref >= (1 << 23) ||
          bref > kOpbMaxRef || o.fv > kOpbFvMask) {
        set_error("pole tree exceeds the program's encodable sizes: leaf run " + std::to_string(o.run) +
                  " (at most 255), live slots " + std::to_string(n_live) + " (" + std::to_string(kMaxSlots) +
                  "), nodes " + std::to_string(base + n_gid) + " (" + std::to_string(1 << kOpbDstBits) +
                  "), adjoint operand " + std::to_string(bref) + " (" + std::to_string(kOpbMaxRef) + ")");
        return TAMI_EUNSUPPORTED;
      }
      ops.push_back({slot[o.dst] | (o.first ? kOpFirst : 0) | (o.leaf ? kOpLeaf : 0) | (fref << kOpRefShift), o.fv});
      opsb.push_back({(base + gid[o.dst]) | (o.first ? kOpbFirst : 0) | (o.leaf ? kOpbLeaf : 0) |
                      (o.run << kOpbRunShift), o.fv | (bref << kOpbRefShift)});
      if (!o.leaf) ++n_inner;
      if (!o.leaf && last_use[o.ref] == (int)p) free_slots.push_back(slot[o.ref]);
    }
    max_slots = std::max(max_slots, n_live);
    g1_node[g] = base;
    node_base += n_gid;
    g1_ops[g] = {begin, (int)ops.size()};
  }
  h.n_ops = (int)ops.size();
  h.n_leaves = (int)leafA.size();
  h.max_depth = m_depth;
  h.n_inner = n_inner;
  h.n_slots = max_slots;
  h.n_nodes = node_base;
  g1_node[g1s.size()] = node_base;
  int ng1rd = 0, ng2cd = 0;
  const int n_mul_ops = (int)ops.size();
  for (auto& g : g1s) ng1rd += (int)g.rd.size();
  for (auto& g : g2s) ng2cd += (int)g.size();
  h.n_g1rd = ng1rd;
  h.n_g2 = (int)g2s.size(); h.n_g2cd = ng2cd;
  h.n_pnode = (int)pnodes.size();
  h.g2_const = g2_const;
  h.max_der = max_der;
  Blob B;
  int n_lm = 0;
  for (int j : repl) for (int l = 0; l < nv; ++l) if (d->alpha[j * nv + l]) ++n_lm;
  h.n_lm = n_lm;
  h.off_alpha = B.reserve(sizeof(double) * N * nv);
  h.off_repl = B.reserve(sizeof(int) * h.n_rep);
  h.off_lm_ptr = B.reserve(sizeof(int) * (h.n_rep + 1));
  h.off_lm_l = B.reserve(sizeof(int) * n_lm);
  h.off_lm_c = B.reserve(sizeof(double) * n_lm);
  h.off_rep_aext = B.reserve(sizeof(double) * h.n_rep);
  h.off_combo_ptr = B.reserve(sizeof(int) * (h.n_combo + 1));
  h.off_combo_j = B.reserve(sizeof(int) * nnz);
  h.off_combo_c = B.reserve(sizeof(double) * nnz);
  h.off_fseg = B.reserve(sizeof(int) * 8 * h.n_fseg);
  h.off_fv = B.reserve(sizeof(int) * 2 * h.n_fv);
  h.off_rden = B.reserve(sizeof(int) * 2 * h.n_rden);
  h.off_cden = B.reserve(sizeof(int) * 2 * h.n_cden);
  h.off_cden_a = B.reserve(sizeof(double) * h.n_cden);
  h.off_cden_xk = B.reserve(sizeof(int) * h.n_cden);
  h.off_xvec = B.reserve(sizeof(double) * h.n_xk * n_ext);
  h.off_g1 = B.reserve(sizeof(int) * 4 * h.n_g1);
  h.off_g1_tgt = B.reserve(sizeof(int) * h.n_g1);
  h.off_g1_node = B.reserve(sizeof(int) * (h.n_g1 + 1));
  h.off_leafA = B.reserve(sizeof(double) * h.n_leaves);
  h.off_g1rd = B.reserve(sizeof(int) * 2 * ng1rd);
  h.off_g2 = B.reserve(sizeof(int) * (h.n_g2 + 1));
  h.off_g2cd = B.reserve(sizeof(int) * 2 * ng2cd);
  h.off_g2cd_p = B.reserve(sizeof(double) * ng2cd);
  h.off_pnode = B.reserve(sizeof(int) * 2 * h.n_pnode);
  h.off_g2node = B.reserve(sizeof(int) * h.n_g2);
  // the two pole-DAG programs last: a forward kernel stages [0, off_opsb), an adjoint [0, off_ops)
  // and [off_opsb, bytes), and a program too large for shared memory is streamed from off_ops
  h.off_ops = B.reserve(sizeof(int) * 2 * h.n_ops);
  h.off_opsb = B.reserve(sizeof(int) * 2 * h.n_ops);
  B.reserve(16);
  h.bytes = (int)B.b.size();

  for (int j = 0; j < N * nv; ++j) B.at<double>(h.off_alpha)[j] = (double)d->alpha[j];
  for (int i = 0; i < h.n_rep; ++i) B.at<int>(h.off_repl)[i] = repl[i];
  {
    int q = 0;
    for (int r = 0; r < h.n_rep; ++r) {
      const int j = repl[r];
      B.at<int>(h.off_lm_ptr)[r] = q;
      for (int l = 0; l < nv; ++l)
        if (d->alpha[j * nv + l]) {
          B.at<int>(h.off_lm_l)[q] = l;
          B.at<double>(h.off_lm_c)[q] = (double)d->alpha[j * nv + l];
          ++q;
        }
      B.at<double>(h.off_rep_aext)[r] = (double)d->alpha[j * nv + m];
    }
    B.at<int>(h.off_lm_ptr)[h.n_rep] = q;
  }
  {
    int k = 0;
    for (int u = 0; u < h.n_combo; ++u) {
      B.at<int>(h.off_combo_ptr)[u] = k;
      for (int j = 0; j < N; ++j)
        if (combos[u][j]) {
          B.at<int>(h.off_combo_j)[k] = j;
          B.at<double>(h.off_combo_c)[k] = (double)combos[u][j];
          ++k;
        }
    }
    B.at<int>(h.off_combo_ptr)[h.n_combo] = k;
  }
  for (int g = 0; g < h.n_fseg; ++g) {
    int* r = B.at<int>(h.off_fseg) + 8 * g;
    r[0] = segs[g].combo; r[1] = segs[g].sigma; r[2] = segs[g].v0; r[3] = segs[g].vk1; r[4] = segs[g].v1;
  }
  for (int v = 0; v < h.n_fv; ++v) {
    int* r = B.at<int>(h.off_fv) + 2 * v;
    r[0] = fvs[v].sign; r[1] = fvs[v].k;
  }
  for (int i = 0; i < h.n_rden; ++i) {
    int* r = B.at<int>(h.off_rden) + 2 * i;
    r[0] = rdens[i]; r[1] = 1;
  }
  for (int i = 0; i < h.n_cden; ++i) {
    int* r = B.at<int>(h.off_cden) + 2 * i;
    r[0] = cdens[i].u; r[1] = cdens[i].sign;
    B.at<double>(h.off_cden_a)[i] = (double)cdens[i].a;
    B.at<int>(h.off_cden_xk)[i] = cdens[i].xk;
  }
  for (int k = 0; k < h.n_xk; ++k)
    for (int q = 0; q < n_ext; ++q) B.at<double>(h.off_xvec)[k * n_ext + q] = (double)xvecs[k][q];
  for (int o = 0; o < h.n_ops; ++o) {
    B.at<int>(h.off_ops)[2 * o] = ops[o].first;
    B.at<int>(h.off_ops)[2 * o + 1] = ops[o].second;
    B.at<int>(h.off_opsb)[2 * o] = opsb[o].first;
    B.at<int>(h.off_opsb)[2 * o + 1] = opsb[o].second;
  }
  for (int g = 0; g <= h.n_g1; ++g) B.at<int>(h.off_g1_node)[g] = g1_node[g];
  for (int i = 0; i < h.n_leaves; ++i) B.at<double>(h.off_leafA)[i] = leafA[i];
  {
    int rdpos = 0;
    for (int g = 0; g < h.n_g1; ++g) {
      int* r = B.at<int>(h.off_g1) + 4 * g;
      r[0] = g1_ops[g].first;
      r[1] = g1_ops[g].second;
      r[2] = rdpos;
      for (auto& pr : g1s[g].rd) {
        B.at<int>(h.off_g1rd)[2 * rdpos] = pr.first;
        B.at<int>(h.off_g1rd)[2 * rdpos + 1] = pr.second;
        ++rdpos;
      }
      r[3] = rdpos;
      B.at<int>(h.off_g1_tgt)[g] = g1s[g].g2;
    }
  }
  {
    int pos = 0;
    for (int g = 0; g < h.n_g2; ++g) {
      B.at<int>(h.off_g2)[g] = pos;
      for (auto& pr : g2s[g]) {
        B.at<int>(h.off_g2cd)[2 * pos] = pr.first;
        B.at<int>(h.off_g2cd)[2 * pos + 1] = pr.second;
        B.at<double>(h.off_g2cd_p)[pos] = (double)pr.second;
        ++pos;
      }
    }
    B.at<int>(h.off_g2)[h.n_g2] = pos;
  }
  for (int k = 0; k < h.n_pnode; ++k) {
    B.at<int>(h.off_pnode)[2 * k] = pnodes[k].first;
    B.at<int>(h.off_pnode)[2 * k + 1] = pnodes[k].second;
  }
  for (int g = 0; g < h.n_g2; ++g) B.at<int>(h.off_g2node)[g] = g2node[g];
  d->blob.swap(B.b);
  {
    std::string why;
    if (!validate_table(h, d->blob.data(), d->blob.size(), &why)) {
      set_error("flattened table failed validation: " + why);
      return TAMI_EUNSUPPORTED;
    }
  }

  // ---- info and the flop model of the kernels' explicit arithmetic
  tami_info& I = d->info;
  I.n_lines = N; I.n_vars = nv;
  I.n_terms = (int64_t)d->terms.size();
  I.n_fermi_factors = nF; I.n_g_factors = nG;
  I.max_der = max_der; I.max_g = max_g;
  I.unique_poles = (int64_t)upoles.size();
  I.unique_dens = (int64_t)udens.size();
  I.n_combos = h.n_combo; I.n_fermi_values = h.n_fv;
  I.n_real_dens = h.n_rden; I.n_cplx_dens = h.n_cden;
  I.n_groups_fixed = h.n_g1; I.n_groups_freq = h.n_g2;
  I.table_bytes = h.bytes;
  I.saved_rows = h.n_rep + 2 * h.n_rep_ext;
  I.n_ext = n_ext;
  // Algorithmic flops of the evaluation, per sample and per (sample, frequency): fma = 2, mul or
  // add = 1, a multiplication by +-1 or an addition to an exact 0 is free (the tables' integer
  // coefficients are mostly +-1; a kernel that multiplies by them anyway does no useful work
  // there), the reciprocal (estimate + one third-order Newton step) 6, the table-driven exponential
  // 8 fma + 3 (e^t - 1: 2 more), cos 30 (reduction 9, series 21), sin 21.  Per frequency the count
  // is that of the imaginary axis; off it the kernels add one more add per complex denominator.
  // Forward sums of the form sum_i c_i y_i (line momenta, energy combinations, pole-DAG nodes) are
  // fma chains from 0, and chains that begin with the same steps share those partial sums: each
  // distinct prefix is counted once, as a compiled kernel evaluates it once.  The reverse passes
  // share nothing (every adjoint differs) and count every step.
  auto unit = [](double c) { return c == 1.0 || c == -1.0; };
  // the derivative polynomial of order k >= 2 (fermi_poly: g h, h - g, the powers of beta, g and h,
  // the Eulerian-number sum)
  auto poly_cost = [](int k) { return k == 2 ? 5.0 : k == 3 ? 9.0 : k == 4 ? 17.0 : 23.0; };
  auto step_cost = [&](bool first, double c) { return first ? (unit(c) ? 0.0 : 1.0) : (unit(c) ? 1.0 : 2.0); };
  struct Prefixes {     // (prefix, variable, operand kind, operand) -> prefix id; cost of the new ones
    std::map<std::tuple<int, int, int, long long>, int> id;
    double flops = 0.0;
    int step(int parent, int var, int kind, long long operand, double cost) {
      const auto r = id.emplace(std::make_tuple(parent, var, kind, operand), (int)id.size() + 1);
      if (r.second) flops += cost;
      return r.first->second;
    }
  };
  auto bits = [](double v) { long long b; std::memcpy(&b, &v, sizeof b); return b; };
  double fl = 0.0;
  fl += 2.0 * 2 * m;                                    // u -> k: one fma per component
  {
    Prefixes mom;                                       // line momenta, both components
    for (int j : repl) {
      int p = 0;
      bool first = true;
      for (int l = 0; l < nv; ++l) {
        const double a = (double)d->alpha[j * nv + l];
        if (a == 0.0) continue;
        p = mom.step(p, l, 0, bits(a), step_cost(first, a));
        first = false;
      }
    }
    fl += 2.0 * mom.flops;
  }
  fl += h.n_rep * (2.0 * 30.0 + 6.0);                   // cos of both components, energy
  const double energy_flops = fl;                       // what a saved-rows adjoint does not redo
  const double ext_grad_flops = h.n_rep_ext * 2.0 * (21.0 + 3.0);   // sin and G = (2t + 4t' cos) sin per component
  Prefixes cmb;                                         // energy combinations (distinct prefixes)
  for (const Vec& c : combos) {
    bool first = true;
    int p = 0;
    for (int j = 0; j < N; ++j)
      if (c[j]) {
        const double cj = (double)c[j];
        p = cmb.step(p, j, 0, bits(cj), step_cost(first, cj));
        first = false;
      }
  }
  fl += cmb.flops;
  for (const Seg& g : segs) {
    fl += 1.0 + 19.0 + (g.sigma < 0 ? 2.0 : 0.0);       // -beta|x|; e^t; e^t - 1
    fl += g.sigma < 0 ? 7.0 : 8.0;                      // D (1 + y, or -(e^t - 1): free), reciprocal, +-y / D
    bool k1 = false;                                    // -beta g h once per segment: every k = 1 value
    for (int v = g.v0; v < g.v1; ++v) {
      const int k = fvs[v].k;
      k1 |= k == 1;
      fl += k <= 1 ? 0.0 : poly_cost(k);
    }
    if (k1) fl += 2.0;
  }
  fl += 6.0 * h.n_rden;                                 // real reciprocals
  double dag_bwd = 0.0;                                 // pole DAG, forward and adjoint
  // groups whose weight is identically zero (every term cancelled): the specialised kernels skip
  // them, weight, products and adjoint alike
  std::vector<char> g1_zero(g1s.size(), 0);
  // The reverse sweep's sums take their first term as an assignment (a copy, free, or a product),
  // every later term as an add or an fma, as the specialised kernels write them: `sum_term` counts
  // one term of a sum whose has-a-value flag is h.
  auto sum_term = [](char& h, double first_cost, double later_cost) {
    const double c = h ? later_cost : first_cost;
    h = 1;
    return c;
  };
  std::vector<char> hfv(fvs.size(), 0);                 // Fermi values whose adjoint has a term
  {
    std::vector<int> flat(2 * opsb.size());
    for (size_t i = 0; i < opsb.size(); ++i) { flat[2 * i] = opsb[i].first; flat[2 * i + 1] = opsb[i].second; }
    const DagPrefixes dp = dag_prefixes(flat.data(), (int)opsb.size(), leafA.data());
    for (size_t g = 0; g < g1s.size(); ++g) g1_zero[g] = dp.node_value[g1_node[g]] < 0;
    for (const DagPrefix& q : dp.p) fl += step_cost(q.parent < 0, q.node ? 2.0 : q.osign * leafA[q.operand]);
    // adjoint, as the specialised kernels walk it: every group root seeded with its weight's adjoint
    // (one mul per group, counted with the groups below; a second seed of the same root is an fma),
    // then the prefixes in reverse creation order: F_y's adjoint += operand x adjoint, a node
    // operand's value gets F_y x adjoint, and the adjoint passes to the parent prefix (each a sum
    // whose first term is a copy or a product)
    std::vector<char> has(dp.p.size(), 0);
    for (int g = 0; g < (int)g1_node.size() - 1 && g < h.n_g1; ++g) {
      const int rp = dp.node_value[g1_node[g]];
      if (rp < 0) continue;
      if (has[rp]) dag_bwd += 1.0;
      has[rp] = 1;
    }
    for (int k = (int)dp.p.size() - 1; k >= 0; --k) {
      if (!has[k]) continue;
      const DagPrefix& q = dp.p[k];
      if (q.node) {
        dag_bwd += sum_term(hfv[q.fv], 1.0, 2.0) + sum_term(has[q.operand], 1.0, 2.0);
      } else {
        const bool u1 = unit(leafA[q.operand]);
        dag_bwd += sum_term(hfv[q.fv], u1 ? 0.0 : 1.0, u1 ? 1.0 : 2.0);
      }
      if (q.parent >= 0) {
        if (has[q.parent]) dag_bwd += 1.0;
        has[q.parent] = 1;
      }
    }
  }
  {
    std::set<int> w2_set;                               // W2 takes its first group weight as a copy
    for (size_t g = 0; g < g1s.size(); ++g) {
      if (g1_zero[g]) continue;
      for (auto& pr : g1s[g].rd) fl += pr.second;       // frequency-independent denominators
      if (!w2_set.insert(g1s[g].g2).second) fl += 1.0;
    }
  }
  I.flops_per_sample = fl;
  I.energy_in_flops_per_sample = fl - energy_flops;
  double ff = 10.0 * h.n_cden;                          // |D|^2, reciprocal, 1/D
  ff += 6.0 * h.n_pnode;                                // complex product per trie node
  // W R accumulated (the R = 1 group is a copy); without it the first group's terms start the
  // sums, two products
  double wr = 0.0;
  {
    bool first = !h.g2_const;
    for (auto& g : g2s) {
      if (g.empty()) continue;
      wr += first ? 2.0 : 4.0;
      first = false;
    }
  }
  ff += wr;
  I.energy_in_flops_per_sample_freq = ff;              // energy input returns the values only
  I.n_dag_ops = h.n_ops;
  I.n_dag_nodes = h.n_nodes;
  I.n_phase2_factors = h.n_g2cd;
  ff += 6.0;                                            // mean and variance sums
  I.flops_per_sample_freq = ff;
  // adjoint: the forward's phase 1 again plus the next derivative of every Fermi value, then per
  // frequency the phase-2 products with the adjoint contractions, then the reverse sweep
  double bl = fl;
  for (const Seg& g : segs) {                           // next derivative of every Fermi value
    bool k1 = false;                                    // -beta g h, shared by the segment's k = 0 values
    for (int v = g.vk1; v < g.v1; ++v) k1 |= fvs[v].k == 1;   // (counted above where k = 1 values use it)
    if (g.vk1 > g.v0 && !k1) bl += 2.0;
    if (k1) bl += 3.0;                                  // -beta d1 (h - g): every k = 1 value's derivative
    for (int v = g.vk1; v < g.v1; ++v)
      if (fvs[v].k != 1) bl += poly_cost(fvs[v].k + 1);
  }
  std::vector<char> hx(combos.size(), 0);              // combinations whose adjoint has a term
  for (const CdKey& c : cdens) bl += sum_term(hx[c.u], 0.0, 1.0);   // cden adjoints into combinations
  for (size_t gi = 0; gi < g1s.size(); ++gi) {
    // the group weight W1 = pv RR, with RR (the product of its real-denominator reciprocals) kept
    // from the forward: the root's adjoint wb RR, and each real denominator's adjoint
    // -wb W1 pw rr (wb W1 once per group, the power a product where it is not 1, one fma or, for the
    // denominator's first term, a product)
    if (g1_zero[gi]) continue;
    const auto& g = g1s[gi];
    if (!g.rd.empty()) bl += 1.0;
    for (auto& pr : g.rd) bl += (pr.second == 1 ? 0.0 : 1.0) + sum_term(hx[rdens[pr.first]], 1.0, 2.0);
    bl += 1.0;
  }
  bl += dag_bwd;
  bl += h.n_rep_ext * 2.0 * 21.0;                       // sin of both components where k_ext enters (series)
  for (auto& g : g2s) for (auto& pr : g) bl += pr.second == 1 ? 0.0 : 1.0;   // p W per group factor
  for (const Seg& g : segs) {                           // +-fvbar P_{k+1} summed per segment into x
    char any = 0;
    double c = 0.0;
    for (int v = g.v0; v < g.v1; ++v)
      if (hfv[v]) c += sum_term(any, 1.0, 2.0);
    if (any) bl += c + sum_term(hx[g.combo], 0.0, 1.0);
  }
  {
    std::vector<char> hE(N, 0);                          // x -> E (the combinations' coefficients)
    for (size_t u = 0; u < combos.size(); ++u) {
      if (!hx[u]) continue;
      for (int j = 0; j < N; ++j)
        if (combos[u][j]) {
          const bool u1 = unit((double)combos[u][j]);
          bl += sum_term(hE[j], u1 ? 0.0 : 1.0, u1 ? 1.0 : 2.0);
        }
    }
  }
  bl += h.n_rep - 1;                                    // E -> mu
  for (int r = 0; r < h.n_rep_ext; ++r)                 // E -> k_ext: (-Ebar a_ext) G per component,
    bl += (r ? 4.0 : 2.0) + (unit((double)d->alpha[repl[r] * nv + m]) ? 0.0 : 1.0);   // the first a product
  I.bwd_flops_per_sample = bl;
  I.fwd_save_flops_per_sample = I.flops_per_sample + ext_grad_flops;
  I.bwd_saved_flops_per_sample = bl - energy_flops - ext_grad_flops;
  double bf = 10.0 * h.n_cden + 2.0;                    // reciprocals, dv/dX accumulated
  for (size_t c = 0; c < cdens.size(); ++c)             // Z, dv/dX (the first starts it), b-adjoint
    bf += 6.0 + (c == 0 ? (unit((double)cdens[c].a) ? 0.0 : 2.0) : (unit((double)cdens[c].a) ? 2.0 : 4.0)) + 4.0;
  bf += 6.0 * h.n_pnode;                                // products (trie nodes)
  {
    std::vector<char> u_set(cdens.size(), 0);          // U += p W R, the first term per factor a product
    for (auto& g : g2s) {
      if (g.empty()) continue;
      bf += 4.0;                                        // Wbar
      for (auto& pr : g) { bf += u_set[pr.first] ? 4.0 : 2.0; u_set[pr.first] = 1; }
    }
  }
  I.bwd_flops_per_sample_freq = bf;
  double fused = bf + 6.0 + wr;                         // the forward's sums, W R accumulated
  I.fused_flops_per_sample_freq = fused;
  return TAMI_OK;
}

// ------------------------------------------------------------------------------ enumerator
namespace {

// Canonical relabelling of a contraction.  up[v] (v < m) is where the up line leaving
// interaction v goes, up[m] is where the incoming external leg enters (m = external slot);
// dn[v] likewise for down lines.  Interaction lines are numbered on first visit: first along
// the external up chain, then, for each numbered line in turn, around the closed up cycle
// through it and the down cycle through it.
bool canonical_code(int m, const int* up, const int* dn, std::vector<int>& code) {
  std::vector<int> newlab(m, -1), visit;
  std::vector<char> upv(m, 0), dnv(m, 0);
  auto mark = [&](int v) { if (newlab[v] < 0) { newlab[v] = (int)visit.size(); visit.push_back(v); } };
  for (int v = up[m]; v != m; v = up[v]) { mark(v); upv[v] = 1; }
  for (size_t q = 0; q < visit.size(); ++q) {
    int i = visit[q];
    if (!upv[i]) for (int v = i;;) { mark(v); upv[v] = 1; v = up[v]; if (v == i) break; }
    if (!dnv[i]) for (int v = i;;) { mark(v); dnv[v] = 1; v = dn[v]; if (v == i) break; }
  }
  if ((int)visit.size() < m) return false;
  code.resize(2 * m + 1);
  code[0] = newlab[up[m]];
  for (int c = 0; c < m; ++c) {
    int old = visit[c];
    code[1 + 2 * c] = up[old] == m ? m : newlab[up[old]];
    code[2 + 2 * c] = newlab[dn[old]];
  }
  return true;
}

struct Labelled {
  std::vector<int8_t> alpha, eps;
  int loops;
};

// Momentum labels of a canonical diagram; false if one-particle reducible or a tadpole.
bool label_code(int m, const std::vector<int>& code, Labelled& L) {
  const int N = 2 * m - 1, nv = m + 1;
  std::vector<int> up(m + 1), dn(m);
  up[m] = code[0];
  for (int c = 0; c < m; ++c) { up[c] = code[1 + 2 * c]; dn[c] = code[2 + 2 * c]; }
  std::vector<int> src, dst;
  int exit_node = -1;
  for (int c = 0; c < m; ++c) {
    if (up[c] == m) exit_node = c;
    else { src.push_back(c); dst.push_back(up[c]); }
  }
  const int n_up = (int)src.size();
  for (int c = 0; c < m; ++c) { src.push_back(c); dst.push_back(dn[c]); }
  if ((int)src.size() != N || exit_node < 0) return false;
  const int root = up[m];
  // BFS tree: dequeue a node, take every line to an unseen node, lines in index order
  std::vector<int> par_line(m, -1), depth(m, -1), order{root};
  depth[root] = 0;
  std::vector<char> is_tree(N, 0);
  for (size_t q = 0; q < order.size(); ++q) {
    int u = order[q];
    for (int j = 0; j < N; ++j) {
      int other;
      if (src[j] == u) other = dst[j];
      else if (dst[j] == u) other = src[j];
      else continue;
      if (depth[other] >= 0) continue;
      depth[other] = depth[u] + 1;
      par_line[other] = j;
      is_tree[j] = 1;
      order.push_back(other);
    }
  }
  std::vector<int> a(N * nv, 0);
  auto parent = [&](int x) { int j = par_line[x]; return src[j] == x ? dst[j] : src[j]; };
  // add `coef` units of flow running from node `from` to node `to` along the tree
  auto route = [&](int from, int to, int var, int coef) {
    int x = from, y = to;
    while (x != y) {
      if (depth[x] >= depth[y]) {           // step x toward the root: flow x -> parent
        int j = par_line[x];
        a[j * nv + var] += (src[j] == x) ? coef : -coef;
        x = parent(x);
      } else {                              // step y toward the root: flow parent -> y
        int j = par_line[y];
        a[j * nv + var] += (dst[j] == y) ? coef : -coef;
        y = parent(y);
      }
    }
  };
  int var = 0;
  for (int j = 0; j < N; ++j) {
    if (is_tree[j]) continue;
    if (var >= m) return false;
    a[j * nv + var] = 1;
    route(dst[j], src[j], var, 1);           // the loop closes from the chord's head back to its tail
    ++var;
  }
  if (var != m) return false;
  route(root, exit_node, m, 1);
  for (int j = 0; j < N; ++j) {
    bool loop = false;
    for (int l = 0; l < m; ++l) loop |= a[j * nv + l] != 0;
    if (!loop) return false;               // a bridge: one-particle reducible
  }
  for (int c = 0; c < m; ++c) {            // momentum transfer through interaction c (up side)
    int jo = -1, ji = -1;
    for (int j = 0; j < n_up; ++j) { if (src[j] == c) jo = j; if (dst[j] == c) ji = j; }
    bool zero = true;
    for (int l = 0; l < nv; ++l) {
      int o = jo >= 0 ? a[jo * nv + l] : (l == m);
      int i = ji >= 0 ? a[ji * nv + l] : (l == m);
      if (o != i) zero = false;
    }
    if (zero) return false;                 // tadpole
  }
  L.alpha.assign(N * nv, 0);
  for (int i = 0; i < N * nv; ++i) L.alpha[i] = (int8_t)a[i];
  L.eps.assign(N * N, 0);
  for (int j = 0; j < N; ++j) {
    int r = j;
    for (int k = 0; k < j && r == j; ++k)
      if (std::equal(a.begin() + j * nv, a.begin() + (j + 1) * nv, a.begin() + k * nv)) r = k;
    L.eps[j * N + r] = 1;
  }
  // closed loops: up cycles avoiding the external slot, and all down cycles
  int loops = 0;
  std::vector<char> seen(m + 1, 0);
  for (int v = up[m]; v != m; v = up[v]) seen[v] = 1;
  for (int c = 0; c < m; ++c) {
    if (seen[c]) continue;
    ++loops;
    for (int v = c; !seen[v]; v = up[v]) seen[v] = 1;
  }
  std::fill(seen.begin(), seen.end(), 0);
  for (int c = 0; c < m; ++c) {
    if (seen[c]) continue;
    ++loops;
    for (int v = c; !seen[v]; v = dn[v]) seen[v] = 1;
  }
  L.loops = loops;
  return true;
}

}  // namespace
}  // namespace tami

using namespace tami;

extern "C" {

const char* tami_last_error(void) { return g_last_error.c_str(); }

int tami_construct_ext(int n_lines, int n_vars, int n_ext, const int8_t* alpha, const int8_t* eps,
                       const uint8_t* var_is_boson, const int32_t* order, double prefactor,
                       tami_diagram** out) {
  return guarded([&]() -> int {
  if (!out || !alpha) { set_error("NULL argument"); return TAMI_EINVAL; }
  *out = nullptr;
  if (n_lines < 1 || n_lines > kMaxLines || n_vars < 2 || n_vars > kMaxVars) {
    set_error("n_lines must be in [1,16] and n_vars in [2,8]");
    return TAMI_EINVAL;
  }
  if (n_ext < 1 || n_ext > kMaxExt || n_ext > n_vars - 1) {
    set_error("n_ext must be in [1,4] and leave at least one summed variable");
    return TAMI_EINVAL;
  }
  const int m = n_vars - n_ext;
  for (int i = 0; i < n_lines * n_vars; ++i)
    if (alpha[i] < -1 || alpha[i] > 1) { set_error("alpha entries must be -1, 0 or 1"); return TAMI_EINVAL; }
  tami_diagram* d = new (std::nothrow) tami_diagram;
  if (!d) { set_error("out of host memory"); return TAMI_ENOMEM; }
  d->N = n_lines;
  d->nv = n_vars;
  d->n_ext = n_ext;
  d->prefactor = prefactor;
  d->alpha.assign(alpha, alpha + n_lines * n_vars);
  d->boson.assign(n_vars, 0);
  if (var_is_boson) for (int l = 0; l < n_vars; ++l) d->boson[l] = var_is_boson[l] ? 1 : 0;
  SymTerm t0;
  for (int j = 0; j < n_lines; ++j) {
    Form g;
    for (int l = 0; l < n_vars; ++l) g.a[l] = alpha[j * n_vars + l];
    for (int k = 0; k < n_lines; ++k) g.e[k] = eps ? eps[j * n_lines + k] : (int8_t)(j == k);
    if (is_zero(g)) { delete d; set_error("a line with zero energy and frequency"); return TAMI_EINVAL; }
    add_factor(t0.G, g, 1);
  }
  std::vector<SymTerm> cur{t0}, nxt;
  std::vector<char> done(m, 0);
  for (int s = 0; s < m; ++s) {
    int p = order ? order[s] : s;
    if (p < 0 || p >= m || done[p]) { delete d; set_error("order must be a permutation of 0..m-1"); return TAMI_EINVAL; }
    done[p] = 1;
    int rc = sum_over(cur, p, n_vars, d->boson, nxt);
    if (rc != TAMI_OK) { delete d; return rc; }
    cur.swap(nxt);
  }
  d->terms.swap(cur);
  int rc = flatten(d);
  if (rc != TAMI_OK) { delete d; return rc; }
  std::vector<SymTerm>().swap(d->terms);   // everything later reads the flattened table
  *out = d;
  return TAMI_OK;
  });
}

int tami_construct(int n_lines, int n_vars, const int8_t* alpha, const int8_t* eps,
                   const uint8_t* var_is_boson, const int32_t* order, double prefactor,
                   tami_diagram** out) {
  return guarded([&]() -> int {
  return tami_construct_ext(n_lines, n_vars, 1, alpha, eps, var_is_boson, order, prefactor, out);
  });
}

int tami_diagram_info(const tami_diagram* d, tami_info* info) {
  if (!d || !info) { set_error("NULL argument"); return TAMI_EINVAL; }
  *info = d->info;
  return TAMI_OK;
}

int tami_enumerate_sigma(int order, int capacity, int8_t* alpha, int8_t* eps, int32_t* code,
                         int32_t* loops, int* n_out) {
  return guarded([&]() -> int {
  if (order < 2 || order > 6 || capacity < 0) { set_error("order must be in [2,6]"); return TAMI_EINVAL; }
  const int m = order, N = 2 * m - 1, nv = m + 1;
  std::set<std::vector<int>> codes;
  std::vector<int> up(m + 1), dn(m), c;
  for (int i = 0; i <= m; ++i) up[i] = i;
  do {
    if (up[m] == m) continue;
    bool fixed = false;
    for (int v = 0; v < m; ++v) fixed |= up[v] == v;
    if (fixed) continue;
    for (int i = 0; i < m; ++i) dn[i] = i;
    do {
      bool f2 = false;
      for (int v = 0; v < m; ++v) f2 |= dn[v] == v;
      if (!f2 && canonical_code(m, up.data(), dn.data(), c)) codes.insert(c);
    } while (std::next_permutation(dn.begin(), dn.end()));
  } while (std::next_permutation(up.begin(), up.end()));
  int n = 0;
  for (const auto& cc : codes) {
    Labelled L;
    if (!label_code(m, cc, L)) continue;
    if (n < capacity) {
      if (alpha) std::copy(L.alpha.begin(), L.alpha.end(), alpha + (size_t)n * N * nv);
      if (eps) std::copy(L.eps.begin(), L.eps.end(), eps + (size_t)n * N * N);
      if (code) std::copy(cc.begin(), cc.end(), code + (size_t)n * (2 * m + 1));
      if (loops) loops[n] = L.loops;
    }
    ++n;
  }
  if (n_out) *n_out = n;
  return TAMI_OK;
  });
}

}  // extern "C"
