// dag_prefixes (tami_host.cpp) on a hand-built pole-DAG program in the adjoint encoding:
//   node 0 = F1*a0 + F2*a1            node 1 = F1*a2 + F2*a1 + F3*a0     (a2 has a0's value)
//   node 2 = F4*node0 + F5*node1
// Node 1 begins with node 0's two steps (leaf a2 equals leaf a0 in value), so its chain extends
// node 0's value: prefixes p0 = F1*a, p1 = p0 + F2*a1 (node 0), p2 = p1 + F3*a0 (node 1),
// p3 = F4*p1, p4 = p3 + F5*p2 (node 2).
// Sign sharing: node 3 = F1*(-2) + F2*(-3) is node 0's chain with every sign flipped, so it lands on
// p0, p1 with sign -1; node 4 = F4*node3 + F5*node1 = -(F4*p1 - F5*p2): its first step is p3 with
// sign -1 and its second a new prefix p5 = p3 + F5*(-p2) (the parent's sign carried into the
// operand's).
// Cancelled operands: node 5 = F1*0 (a leaf whose terms cancelled) is identically zero and gets no
// prefix; node 6 = F4*node5 + F5*node1 skips its zero first step, so its value is a new first step
// p6 = F5*p2.  Built and run by tests/test_host_harness_cpu.py; no GPU.
#include <cstdio>
#include <vector>

#include "tami_internal.h"

using namespace tami;

static int op(int dst, bool first, bool leaf) { return dst | (first ? kOpbFirst : 0) | (leaf ? kOpbLeaf : 0); }
static int fv(int f, int ref) { return f | (ref << kOpbRefShift); }

int main() {
  const double leafA[6] = {2.0, 3.0, 2.0, -2.0, -3.0, 0.0};
  const std::vector<int> ops = {op(0, true, true), fv(1, 0),  op(0, false, true), fv(2, 1),
                                op(1, true, true), fv(1, 2),  op(1, false, true), fv(2, 1),  op(1, false, true), fv(3, 0),
                                op(2, true, false), fv(4, 0), op(2, false, false), fv(5, 1),
                                op(3, true, true), fv(1, 3),  op(3, false, true), fv(2, 4),
                                op(4, true, false), fv(4, 3), op(4, false, false), fv(5, 1),
                                op(5, true, true), fv(1, 5),
                                op(6, true, false), fv(4, 5), op(6, false, false), fv(5, 1)};
  const DagPrefixes dp = dag_prefixes(ops.data(), (int)ops.size() / 2, leafA);
  int fails = 0;
  auto expect = [&](bool ok, const char* what) { std::printf("%s %s\n", ok ? "ok" : "FAIL", what); fails += !ok; };
  expect(dp.p.size() == 7, "seven distinct prefixes for fourteen ops");
  const std::vector<char> created = {1, 1, 0, 0, 1, 1, 1, 0, 0, 0, 1, 0, 0, 1};
  expect(std::vector<char>(dp.op_new.begin(), dp.op_new.end()) == created, "ops that create a prefix");
  expect(dp.op_prefix == std::vector<int>({0, 1, 0, 1, 2, 3, 4, 0, 1, 3, 5, -1, -1, 6}), "the prefix each op lands on");
  expect(std::vector<int>(dp.op_sign.begin(), dp.op_sign.end()) ==
             std::vector<int>({1, 1, 1, 1, 1, 1, 1, -1, -1, -1, -1, 1, 1, 1}),
         "the sign each op's partial sum takes");
  expect(dp.node_value == std::vector<int>({1, 2, 4, 1, 5, -1, 6}), "node values (-1: identically zero)");
  expect(std::vector<int>(dp.node_sign.begin(), dp.node_sign.end()) == std::vector<int>({1, 1, 1, -1, -1, 1, 1}),
         "node signs");
  expect(dp.p[6].parent == -1 && dp.p[6].fv == 5 && dp.p[6].node == 1 && dp.p[6].operand == 2 && dp.p[6].osign == 1,
         "a zero first step skipped: the next step starts the chain");
  expect(dp.p[2].parent == 1 && dp.p[2].node == 0 && dp.p[2].fv == 3, "node 1 extends node 0's value");
  expect(dp.p[3].parent == -1 && dp.p[3].node == 1 && dp.p[3].operand == 1, "node operand = its value prefix");
  expect(dp.p[4].parent == 3 && dp.p[4].operand == 2 && dp.p[4].osign == 1, "second node operand");
  expect(dp.p[0].osign == 1 && dp.p[1].osign == 1 && dp.p[3].osign == 1, "positive chains keep their operands' signs");
  expect(dp.p[5].parent == 3 && dp.p[5].fv == 5 && dp.p[5].node == 1 && dp.p[5].operand == 2 && dp.p[5].osign == -1,
         "a flipped chain's next step: the parent's sign carried into the operand");
  std::printf("%d failures\n", fails);
  return fails ? 1 : 0;
}
