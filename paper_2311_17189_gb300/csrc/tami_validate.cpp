// Host-side validation of a flattened term table before it is uploaded: every index the kernels
// read is checked against the size of what it indexes, the segment and group ranges against each
// other, and both pole-DAG programs against their slot liveness (no value read before it is
// written, every group ending on its root).  A table that fails is never uploaded.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "tami_internal.h"

namespace tami {
namespace {

struct Reader {
  const unsigned char* b;
  size_t size;
  bool ok = true;
  std::string why;
  template <typename T>
  const T* at(int off, size_t count, const char* what) {
    if (!ok) return nullptr;
    if (off < 0 || (off & 15) != 0 || (size_t)off + sizeof(T) * count > size) {
      ok = false;
      why = std::string("section out of the blob: ") + what;
      return nullptr;
    }
    return reinterpret_cast<const T*>(b + off);
  }
  bool fail(const std::string& w) {
    if (ok) { ok = false; why = w; }
    return false;
  }
};

bool in(long long v, long long lo, long long hi) { return v >= lo && v < hi; }

}  // namespace

bool validate_table(const TableHeader& h, const unsigned char* blob, size_t size, std::string* why) {
  // every section but the two programs lies in [0, off_ops); the programs are [off_ops, off_opsb)
  // and [off_opsb, bytes) (the kernels stage these ranges by themselves)
  const size_t prog = (size_t)h.off_ops;
  Reader R{blob, prog <= size ? prog : 0};
  auto bad = [&](const std::string& w) { R.fail(w); };
  if ((size_t)h.bytes != size) bad("header size differs from the blob");
  const size_t prog_bytes = (8 * (size_t)std::max(h.n_ops, 0) + 15) & ~size_t(15);
  if (h.off_ops < 0 || (h.off_ops & 15) != 0 || (size_t)h.off_opsb != prog + prog_bytes ||
      (size_t)h.bytes != prog + 2 * prog_bytes + 16)
    bad("pole-DAG programs are not the last sections");
  if (!in(h.N, 1, kMaxLines + 1) || !in(h.nv, 2, kMaxVars + 1) || !in(h.n_ext, 1, kMaxExt + 1) ||
      h.m != h.nv - h.n_ext || h.m < 1)
    bad("line or variable count");
  if (!in(h.n_xk, 1, kMaxCplxDens + 2) || (h.n_ext == 1 && h.n_xk != 1)) bad("external-coefficient vectors");
  if (h.n_rep_ext < 0 || h.n_rep_ext > h.n_rep || h.n_rep > h.N) bad("representative lines");
  if (h.n_combo > kMaxCombos || h.n_fv > kMaxFermiValues || h.n_rden > kMaxRealDens || h.n_cden > kMaxCplxDens ||
      h.n_pnode > kMaxProdNodes || h.n_slots > kMaxSlots || h.max_der > kMaxDer || h.max_der < 0)
    bad("a count above the kernels' capacities");
  if (!R.ok) { *why = R.why; return false; }

  const int* repl = R.at<int>(h.off_repl, h.n_rep, "repl");
  const int* lm_ptr = R.at<int>(h.off_lm_ptr, h.n_rep + 1, "lm_ptr");
  const int* lm_l = R.at<int>(h.off_lm_l, h.n_lm, "lm_l");
  const int* combo_ptr = R.at<int>(h.off_combo_ptr, h.n_combo + 1, "combo_ptr");
  const int* combo_j = R.at<int>(h.off_combo_j, h.combo_nnz, "combo_j");
  const int* fseg = R.at<int>(h.off_fseg, 8 * (size_t)h.n_fseg, "fseg");
  const int* fvr = R.at<int>(h.off_fv, 2 * (size_t)h.n_fv, "fv");
  const int* rden = R.at<int>(h.off_rden, 2 * (size_t)h.n_rden, "rden");
  const int* cden = R.at<int>(h.off_cden, 2 * (size_t)h.n_cden, "cden");
  const int* cden_xk = R.at<int>(h.off_cden_xk, h.n_cden, "cden_xk");
  const double* xvec = R.at<double>(h.off_xvec, (size_t)h.n_xk * h.n_ext, "xvec");
  const int* g1 = R.at<int>(h.off_g1, 4 * (size_t)h.n_g1, "g1");
  const int* g1_tgt = R.at<int>(h.off_g1_tgt, h.n_g1, "g1_tgt");
  Reader RP{blob, size};
  const int* ops = RP.at<int>(h.off_ops, 2 * (size_t)h.n_ops, "ops");
  const int* opsb = RP.at<int>(h.off_opsb, 2 * (size_t)h.n_ops, "opsb");
  if (!RP.ok) bad(RP.why);
  const int* g1_node = R.at<int>(h.off_g1_node, h.n_g1 + 1, "g1_node");
  R.at<double>(h.off_leafA, h.n_leaves, "leafA");
  const int* g1rd = R.at<int>(h.off_g1rd, 2 * (size_t)h.n_g1rd, "g1rd");
  const int* g2 = R.at<int>(h.off_g2, h.n_g2 + 1, "g2");
  const int* g2cd = R.at<int>(h.off_g2cd, 2 * (size_t)h.n_g2cd, "g2cd");
  const int* pnode = R.at<int>(h.off_pnode, 2 * (size_t)h.n_pnode, "pnode");
  const int* g2node = R.at<int>(h.off_g2node, h.n_g2, "g2node");
  if (!R.ok) { *why = R.why; return false; }

  std::vector<char> computed(h.N, 0);
  for (int r = 0; r < h.n_rep; ++r) {
    if (!in(repl[r], 0, h.N)) bad("representative line index");
    else computed[repl[r]] = 1;
    if (lm_ptr[r] > lm_ptr[r + 1]) bad("label ranges");
  }
  if (lm_ptr[0] != 0 || lm_ptr[h.n_rep] != h.n_lm) bad("label ranges");
  for (int q = 0; q < h.n_lm; ++q) if (!in(lm_l[q], 0, h.nv)) bad("label variable index");
  if (combo_ptr[0] != 0 || combo_ptr[h.n_combo] != h.combo_nnz) bad("combination ranges");
  for (int u = 0; u < h.n_combo; ++u) if (combo_ptr[u] > combo_ptr[u + 1]) bad("combination ranges");
  for (int q = 0; q < h.combo_nnz; ++q)
    if (!in(combo_j[q], 0, h.N) || !computed[combo_j[q]]) bad("combination reads an energy that is not computed");
  // Fermi segments: contiguous, Bose-type first, k = 0 values before k >= 1
  int v = 0;
  for (int s = 0; s < h.n_fseg; ++s) {
    const int* g = fseg + 8 * s;
    if (!in(g[0], 0, h.n_combo)) bad("segment combination");
    if (g[1] != (s < h.n_fseg_bose ? -1 : 1)) bad("segment sigma order");
    if (g[2] != v || g[2] > g[3] || g[3] > g[4] || g[4] > h.n_fv) bad("segment value ranges");
    for (int i = g[2]; i < g[4] && i < h.n_fv; ++i) {
      const int sign = fvr[2 * i], k = fvr[2 * i + 1];
      if ((sign != 1 && sign != -1) || !in(k, 0, h.max_der + 1) || ((i < g[3]) != (k == 0))) bad("Fermi value record");
    }
    v = g[4];
  }
  if (v != h.n_fv) bad("segments do not cover the Fermi values");
  for (int i = 0; i < h.n_rden; ++i) if (!in(rden[2 * i], 0, h.n_combo)) bad("real denominator combination");
  for (int i = 0; i < h.n_cden; ++i)
    if (!in(cden[2 * i], 0, h.n_combo) || (cden[2 * i + 1] != 1 && cden[2 * i + 1] != -1) || !in(cden_xk[i], 0, h.n_xk))
      bad("complex denominator");
  if (h.n_ext == 1 && xvec[0] != 1.0) bad("external-coefficient vector of a one-external table");
  // phase-1 groups and both pole-DAG programs
  if (g1_node[0] != 0 || g1_node[h.n_g1] != h.n_nodes || h.n_nodes > (1 << kOpbDstBits)) bad("DAG node ranges");
  int op_end = 0, rd_end = 0;
  std::vector<char> wf(kMaxSlots), wb(h.n_nodes > 0 ? h.n_nodes : 1);
  for (int gi = 0; gi < h.n_g1 && R.ok; ++gi) {
    const int o0 = g1[4 * gi], o1 = g1[4 * gi + 1], r0 = g1[4 * gi + 2], r1 = g1[4 * gi + 3];
    if (o0 != op_end || o1 <= o0 || o1 > h.n_ops || r0 != rd_end || r1 < r0 || r1 > h.n_g1rd) bad("group ranges");
    if (!in(g1_tgt[gi], 0, h.n_g2) || (gi > 0 && g1_tgt[gi] < g1_tgt[gi - 1])) bad("group target");
    if (g1_node[gi] >= g1_node[gi + 1]) bad("group without DAG nodes");
    if (!R.ok) break;
    op_end = o1;
    rd_end = r1;
    for (int q = r0; q < r1; ++q)
      if (!in(g1rd[2 * q], 0, h.n_rden) || g1rd[2 * q + 1] < 1) bad("real denominator power");
    std::fill(wf.begin(), wf.end(), 0);
    std::fill(wb.begin(), wb.end(), 0);
    int last_dst = -1;
    for (int o = o0; o < o1; ++o) {
      const int x = ops[2 * o], y = ops[2 * o + 1];
      const int dst = x & kOpDstMask, ref = x >> kOpRefShift;
      const bool leaf = x & kOpLeaf, first = x & kOpFirst;
      if (!in(y, 0, h.n_fv) || !in(dst, 0, h.n_slots)) { bad("forward op operand"); break; }
      if (leaf ? !in(ref, 0, h.n_leaves) : !(in(ref, 0, h.n_slots) && wf[ref])) { bad("forward op reads an unset slot"); break; }
      if (!first && !wf[dst]) { bad("forward op accumulates into an unset slot"); break; }
      wf[dst] = 1;
      last_dst = dst;
      const int xb = opsb[2 * o], yb = opsb[2 * o + 1];
      const int bd = xb & kOpbDstMask, br = yb >> kOpbRefShift, run = (xb >> kOpbRunShift) & 255;
      const bool bl = xb & kOpbLeaf, bf = xb & kOpbFirst;
      if ((yb & kOpbFvMask) != y || yb < 0 || xb < 0 || bl != leaf || bf != first || !in(bd, g1_node[gi], g1_node[gi + 1])) { bad("adjoint op"); break; }
      if (bl ? !in(br, 0, h.n_leaves) : !(in(br, g1_node[gi], g1_node[gi + 1]) && wb[br])) { bad("adjoint op reads an unset node"); break; }
      if (!bf && !wb[bd]) { bad("adjoint op accumulates into an unset node"); break; }
      if (run > 0) {   // the run's leaf edges are the run - 1 ops before this one, all into bd
        if (!bl || o - run + 1 < o0) { bad("leaf run"); break; }
        for (int i = 1; i < run; ++i) {
          const int xp = opsb[2 * (o - i)];
          if (!(xp & kOpbLeaf) || (xp & kOpbDstMask) != bd) { bad("leaf run"); break; }
        }
      }
      wb[bd] = 1;
    }
    if (R.ok && !wb[g1_node[gi]]) bad("group root never written");
    if (R.ok && (last_dst < 0 || (opsb[2 * (o1 - 1)] & kOpbDstMask) != g1_node[gi])) bad("group does not end on its root");
  }
  if (R.ok && (op_end != h.n_ops || rd_end != h.n_g1rd)) bad("groups do not cover the program");
  // phase 2
  if (g2[0] != 0 || g2[h.n_g2] != h.n_g2cd) bad("phase-2 group ranges");
  for (int k = 0; k < h.n_pnode; ++k)
    if (!in(pnode[2 * k], 0, h.n_cden + k) || !in(pnode[2 * k + 1], 0, h.n_cden)) bad("product node");
  for (int hg = 0; hg < h.n_g2 && R.ok; ++hg) {
    if (g2[hg] > g2[hg + 1]) bad("phase-2 group ranges");
    const bool empty = g2[hg] == g2[hg + 1];
    if (empty != (hg == 0 && h.g2_const == 1)) bad("frequency-free group not first");
    if (empty ? g2node[hg] != -1 : !in(g2node[hg], 0, h.n_cden + h.n_pnode)) bad("group product node");
    for (int q = g2[hg]; q < g2[hg + 1]; ++q)
      if (!in(g2cd[2 * q], 0, h.n_cden) || g2cd[2 * q + 1] < 1) bad("complex denominator power");
  }
  if (!R.ok) *why = R.why;
  return R.ok;
}

}  // namespace tami
