// Graph representation of a self-energy diagram and its momentum labelling (Sec. 2.5: a plain
// 4-column file "source target B/F spin" per line, read_graph / label_graph / graph_to_R0).
//
// Convention for a self-energy graph.  Vertices are 0..V-1.  Fermionic lines (column 3 = 1) are
// directed source -> target along the particle flow; bosonic lines (column 3 = 0) are
// instantaneous interaction lines joining two vertices and carry no propagator.  One vertex X
// (the external vertex) has exactly one outgoing and one incoming fermionic line -- the amputated
// external legs -- and no bosonic line; every other vertex has one incoming and one outgoing
// fermionic line and one bosonic line.  The spin column is carried along, not used for labels.
//
// Labelling.  The two ends of a bosonic line form one node (momentum is conserved by the pair,
// the interaction's transfer being free).  Internal fermionic lines, in file order, are the
// rows of alpha.  A spanning tree grows breadth first from the node the incoming leg enters; for
// each node taken from the queue the lines are scanned in row order and every line to a new node
// joins the tree.  The other lines carry one loop variable each (in row order); a tree line
// carries the loops whose cycle passes through it; the external momentum runs along the tree
// path from the entry node to the node the outgoing leg leaves.  Rows with equal labels share one
// base energy (eps).  Closed fermion loops are counted for the sign (-1)^F.
#include <algorithm>
#include <cmath>
#include <vector>

#include "tami_internal.h"

namespace tami {
namespace {

struct GraphLabels {
  int N = 0, nv = 0, loops = 0;
  std::vector<int8_t> alpha, eps;
  std::vector<int> row_line;   // input line index of each row
};

int label_graph_impl(const int32_t* ed, int n_edges, GraphLabels& G) {
  if (!ed || n_edges < 3) { set_error("need at least 3 lines"); return TAMI_EINVAL; }
  int V = 0;
  for (int i = 0; i < n_edges; ++i) {
    const int32_t s = ed[4 * i], t = ed[4 * i + 1], f = ed[4 * i + 2];
    if (s < 0 || t < 0 || (f != 0 && f != 1)) { set_error("line " + std::to_string(i) + ": bad vertex or B/F flag"); return TAMI_EINVAL; }
    V = std::max(V, std::max(s, t) + 1);
  }
  std::vector<int> fin(V, 0), fout(V, 0), nb(V, 0), bpartner(V, -1);
  for (int i = 0; i < n_edges; ++i) {
    const int s = ed[4 * i], t = ed[4 * i + 1];
    if (ed[4 * i + 2] == 1) { fout[s]++; fin[t]++; }
    else {
      if (s == t) { set_error("bosonic line with both ends on one vertex"); return TAMI_EINVAL; }
      nb[s]++; nb[t]++; bpartner[s] = t; bpartner[t] = s;
    }
  }
  int X = -1;
  for (int v = 0; v < V; ++v) {
    if (fin[v] != 1 || fout[v] != 1) { set_error("vertex " + std::to_string(v) + " needs one fermionic line in and one out"); return TAMI_EINVAL; }
    if (nb[v] == 0) {
      if (X >= 0) { set_error("more than one vertex without a bosonic line"); return TAMI_EINVAL; }
      X = v;
    } else if (nb[v] != 1) {
      set_error("vertex " + std::to_string(v) + " has more than one bosonic line");
      return TAMI_EINVAL;
    }
  }
  if (X < 0) { set_error("no external vertex (one without a bosonic line)"); return TAMI_EINVAL; }
  // nodes: bosonic pairs
  std::vector<int> node(V, -1);
  int n_nodes = 0;
  for (int v = 0; v < V; ++v) {
    if (v == X || node[v] >= 0) continue;
    node[v] = node[bpartner[v]] = n_nodes++;
  }
  // internal fermionic lines in file order; the legs
  std::vector<int> src, dst;
  int entry = -1, exit_node = -1;
  for (int i = 0; i < n_edges; ++i) {
    if (ed[4 * i + 2] != 1) continue;
    const int s = ed[4 * i], t = ed[4 * i + 1];
    if (s == X && t == X) { set_error("external legs joined to each other"); return TAMI_EINVAL; }
    if (s == X) { entry = node[t]; continue; }
    if (t == X) { exit_node = node[s]; continue; }
    src.push_back(node[s]);
    dst.push_back(node[t]);
    G.row_line.push_back(i);
  }
  const int N = (int)src.size();
  const int m = N - n_nodes + 1;
  if (N < 1 || N > kMaxLines || m < 1 || m + 1 > kMaxVars) { set_error("unsupported number of lines or loops"); return TAMI_EUNSUPPORTED; }
  const int nv = m + 1;
  std::vector<int> depth(n_nodes, -1), par(n_nodes, -1), queue{entry};
  std::vector<char> tree(N, 0);
  depth[entry] = 0;
  for (size_t q = 0; q < queue.size(); ++q) {
    const int u = queue[q];
    for (int j = 0; j < N; ++j) {
      int o = src[j] == u ? dst[j] : (dst[j] == u ? src[j] : -1);
      if (o < 0 || depth[o] >= 0) continue;
      depth[o] = depth[u] + 1;
      par[o] = j;
      tree[j] = 1;
      queue.push_back(o);
    }
  }
  if ((int)queue.size() != n_nodes) { set_error("graph is not connected"); return TAMI_EINVAL; }
  std::vector<int> a(N * nv, 0);
  auto up = [&](int x) { const int j = par[x]; return src[j] == x ? dst[j] : src[j]; };
  auto flow = [&](int from, int to, int var) {   // one unit of flow from -> to along the tree
    int x = from, y = to;
    while (x != y) {
      if (depth[x] >= depth[y]) { const int j = par[x]; a[j * nv + var] += src[j] == x ? 1 : -1; x = up(x); }
      else { const int j = par[y]; a[j * nv + var] += dst[j] == y ? 1 : -1; y = up(y); }
    }
  };
  int var = 0;
  for (int j = 0; j < N; ++j) {
    if (tree[j]) continue;
    a[j * nv + var] = 1;
    flow(dst[j], src[j], var);
    ++var;
  }
  if (var != m) { set_error("loop count mismatch"); return TAMI_EINVAL; }
  flow(entry, exit_node, m);
  for (int v : a) if (v < -1 || v > 1) { set_error("labels outside {-1,0,1}"); return TAMI_EUNSUPPORTED; }
  G.N = N;
  G.nv = nv;
  G.alpha.assign(N * nv, 0);
  for (int i = 0; i < N * nv; ++i) G.alpha[i] = (int8_t)a[i];
  G.eps.assign(N * N, 0);
  for (int j = 0; j < N; ++j) {
    int r = j;
    for (int k = 0; k < j && r == j; ++k)
      if (std::equal(a.begin() + j * nv, a.begin() + (j + 1) * nv, a.begin() + k * nv)) r = k;
    G.eps[j * N + r] = 1;
  }
  // closed fermion loops: cycles of the fermionic successor map that avoid X
  std::vector<int> next(V, -1);
  for (int i = 0; i < n_edges; ++i)
    if (ed[4 * i + 2] == 1) next[ed[4 * i]] = ed[4 * i + 1];
  std::vector<char> seen(V, 0);
  for (int v = next[X]; v != X && v >= 0 && !seen[v]; v = next[v]) seen[v] = 1;
  int loops = 0;
  for (int v = 0; v < V; ++v) {
    if (seen[v] || v == X) continue;
    ++loops;
    for (int w = v; !seen[w]; w = next[w]) seen[w] = 1;
  }
  G.loops = loops;
  return TAMI_OK;
}

}  // namespace
}  // namespace tami

using namespace tami;

extern "C" {

int tami_label_graph(const int32_t* edges, int n_edges, int capacity_lines, int8_t* alpha, int8_t* eps,
                     int32_t* row_line, int* n_lines, int* n_vars, int* loops) {
  return guarded([&]() -> int {
  GraphLabels G;
  int rc = label_graph_impl(edges, n_edges, G);
  if (rc) return rc;
  if (n_lines) *n_lines = G.N;
  if (n_vars) *n_vars = G.nv;
  if (loops) *loops = G.loops;
  if (capacity_lines < G.N) return TAMI_OK;   // sizes only
  if (alpha) std::copy(G.alpha.begin(), G.alpha.end(), alpha);
  if (eps) std::copy(G.eps.begin(), G.eps.end(), eps);
  if (row_line) std::copy(G.row_line.begin(), G.row_line.end(), row_line);
  return TAMI_OK;
  });
}

int tami_construct_from_graph(const int32_t* edges, int n_edges, double prefactor, tami_diagram** out) {
  return guarded([&]() -> int {
  GraphLabels G;
  int rc = label_graph_impl(edges, n_edges, G);
  if (rc) return rc;
  return tami_construct(G.N, G.nv, G.alpha.data(), G.eps.data(), nullptr, nullptr, prefactor, out);
  });
}

}  // extern "C"
