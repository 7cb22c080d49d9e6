// dag_prefixes (tami_host.cpp) on a hand-built pole-DAG program in the adjoint encoding:
//   node 0 = F1*a0 + F2*a1            node 1 = F1*a2 + F2*a1 + F3*a0     (a2 has a0's value)
//   node 2 = F4*node0 + F5*node1
// Node 1 begins with node 0's two steps (leaf a2 equals leaf a0 in value), so its chain extends
// node 0's value: prefixes p0 = F1*a, p1 = p0 + F2*a1 (node 0), p2 = p1 + F3*a0 (node 1),
// p3 = F4*p1, p4 = p3 + F5*p2 (node 2).  Built and run by tests/test_host_harness_cpu.py; no GPU.
#include <cstdio>
#include <vector>

#include "tami_internal.h"

using namespace tami;

static int op(int dst, bool first, bool leaf) { return dst | (first ? kOpbFirst : 0) | (leaf ? kOpbLeaf : 0); }
static int fv(int f, int ref) { return f | (ref << kOpbRefShift); }

int main() {
  const double leafA[3] = {2.0, 3.0, 2.0};
  const std::vector<int> ops = {op(0, true, true), fv(1, 0),  op(0, false, true), fv(2, 1),
                                op(1, true, true), fv(1, 2),  op(1, false, true), fv(2, 1),  op(1, false, true), fv(3, 0),
                                op(2, true, false), fv(4, 0), op(2, false, false), fv(5, 1)};
  const DagPrefixes dp = dag_prefixes(ops.data(), (int)ops.size() / 2, leafA);
  int fails = 0;
  auto expect = [&](bool ok, const char* what) { std::printf("%s %s\n", ok ? "ok" : "FAIL", what); fails += !ok; };
  expect(dp.p.size() == 5, "five distinct prefixes for seven ops");
  const std::vector<char> created = {1, 1, 0, 0, 1, 1, 1};
  expect(std::vector<char>(dp.op_new.begin(), dp.op_new.end()) == created, "ops that create a prefix");
  expect(dp.op_prefix == std::vector<int>({0, 1, 0, 1, 2, 3, 4}), "the prefix each op lands on");
  expect(dp.node_value == std::vector<int>({1, 2, 4}), "node values");
  expect(dp.p[2].parent == 1 && dp.p[2].node == 0 && dp.p[2].fv == 3, "node 1 extends node 0's value");
  expect(dp.p[3].parent == -1 && dp.p[3].node == 1 && dp.p[3].operand == 1, "node operand = its value prefix");
  expect(dp.p[4].parent == 3 && dp.p[4].operand == 2, "second node operand");
  std::printf("%d failures\n", fails);
  return fails ? 1 : 0;
}
