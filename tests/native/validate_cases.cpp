// Corrupts one field of a real flattened table at a time and checks that the host-side validator
// refuses it (and accepts the untouched table).  Built and run by tests/test_validate_cpu.py.
#include <cstdio>
#include <cstring>
#include <functional>
#include <string>
#include <vector>

#include "tami_internal.h"

using namespace tami;

int main() {
  // order-4 self-energy diagram with the largest flat table (canonical code 0 1 1 4 2 3 3 2 0)
  int n = 0;
  tami_enumerate_sigma(4, 0, nullptr, nullptr, nullptr, nullptr, &n);
  const int N = 7, nv = 5;
  std::vector<int8_t> alpha((size_t)n * N * nv), eps((size_t)n * N * N);
  std::vector<int32_t> code((size_t)n * 9);
  tami_enumerate_sigma(4, n, alpha.data(), eps.data(), code.data(), nullptr, &n);
  const int want[9] = {0, 1, 1, 4, 2, 3, 3, 2, 0};
  int idx = -1;
  for (int i = 0; i < n && idx < 0; ++i) if (!std::memcmp(&code[(size_t)i * 9], want, sizeof want)) idx = i;
  tami_diagram* d = nullptr;
  if (idx < 0 || tami_construct(N, nv, &alpha[(size_t)idx * N * nv], &eps[(size_t)idx * N * N], nullptr, nullptr,
                                1.0, &d)) { std::printf("FAIL construct\n"); return 1; }
  const TableHeader h0 = d->hdr;
  const std::vector<unsigned char> b0 = d->blob;
  std::string why;
  if (!tami::validate_table(h0, b0.data(), b0.size(), &why)) { std::printf("FAIL clean table: %s\n", why.c_str()); return 1; }
  auto I = [](std::vector<unsigned char>& b, int off, int k) { return reinterpret_cast<int*>(b.data() + off) + k; };
  struct Case { const char* name; std::function<void(TableHeader&, std::vector<unsigned char>&)> f; };
  std::vector<Case> cases = {
    {"combination reads a line out of range", [&](TableHeader& h, auto& b) { *I(b, h.off_combo_j, 0) = h.N; }},
    {"segment range past the values", [&](TableHeader& h, auto& b) { *I(b, h.off_fseg, 8 * (h.n_fseg - 1) + 4) = h.n_fv + 1; }},
    {"Fermi value with k above max_der", [&](TableHeader& h, auto& b) { *I(b, h.off_fv, 2 * (h.n_fv - 1) + 1) = h.max_der + 1; }},
    {"forward op reads an unset slot", [&](TableHeader& h, auto& b) {
       int* x = I(b, h.off_ops, 0); *x = (*x & ~kOpLeaf & ~(-1 << kOpRefShift)) | ((h.n_slots - 1) << kOpRefShift); }},
    {"forward op slot beyond n_slots", [&](TableHeader& h, auto& b) { int* x = I(b, h.off_ops, 0); *x = (*x & ~kOpDstMask) | kOpDstMask; }},
    {"adjoint op writes outside its group", [&](TableHeader& h, auto& b) {
       int* x = I(b, h.off_opsb, 0); *x = (*x & ~kOpbDstMask) | (h.n_nodes - 1); }},
    {"leaf run longer than the node's leaves", [&](TableHeader& h, auto& b) {
       for (int o = 0; o < h.n_ops; ++o) { int* x = I(b, h.off_opsb, 2 * o);
         if ((*x >> kOpbRunShift) & 255) { *x = (*x & ~(255 << kOpbRunShift)) | (200 << kOpbRunShift); break; } } }},
    {"Fermi value index out of range", [&](TableHeader& h, auto& b) { *I(b, h.off_ops, 1) = h.n_fv; }},
    {"product node refers forward", [&](TableHeader& h, auto& b) { if (h.n_pnode) *I(b, h.off_pnode, 0) = h.n_cden; }},
    {"group product node out of range", [&](TableHeader& h, auto& b) { *I(b, h.off_g2node, h.n_g2 - 1) = h.n_cden + h.n_pnode; }},
    {"phase-1 group ranges overlap", [&](TableHeader& h, auto& b) { *I(b, h.off_g1, 0) = 1; }},
    {"slot count above capacity", [&](TableHeader& h, auto&) { h.n_slots = kMaxSlots + 1; }},
    {"section past the blob end", [&](TableHeader& h, auto&) { h.off_g2node = h.bytes; }},
    {"section inside the pole-DAG programs", [&](TableHeader& h, auto&) { h.off_g2node = h.off_ops; }},
    {"adjoint program overlapping the forward one", [&](TableHeader& h, auto&) { h.off_opsb = h.off_ops; }},
    {"external-coefficient vector index out of range", [&](TableHeader& h, auto& b) { *I(b, h.off_cden_xk, 0) = h.n_xk; }},
    {"external count inconsistent with the variables", [&](TableHeader& h, auto&) { h.n_ext = 2; }},
  };
  int failures = 0;
  for (auto& c : cases) {
    TableHeader h = h0;
    std::vector<unsigned char> b = b0;
    c.f(h, b);
    const bool ok = tami::validate_table(h, b.data(), b.size(), &why);
    std::printf("%s: %s%s\n", ok ? "FAIL accepted" : "refused", c.name, ok ? "" : (" (" + why + ")").c_str());
    failures += ok;
  }
  tami_destroy(d);
  return failures ? 1 : 0;
}
