// Internal layout of libtami: the symbolic solution kept on the host and the flattened
// device term table the kernels read.  Not part of the public ABI.
#pragma once

#include <array>
#include <cmath>
#include <cstdint>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/tami.h"

namespace tami {

constexpr int kMaxLines = TAMI_MAX_LINES;
constexpr int kMaxVars = TAMI_MAX_VARS;
constexpr int kMaxExt = TAMI_MAX_EXT;

// Per-thread capacities of the evaluation kernels (checked at flatten time).
constexpr int kMaxCombos = 128;
constexpr int kMaxFermiValues = 256;
constexpr int kMaxRealDens = 128;
constexpr int kMaxCplxDens = 64;
constexpr int kMaxProdNodes = 128;   // phase-2 product nodes beyond the reciprocals themselves
constexpr int kMaxDer = 5;
constexpr int kMaxDepth = kMaxVars;   // pole-tree depth = number of summed variables

// Pole-tree programs (see flatten): one op per edge, v[dst] = F * (leaf ? A[ref] : v[ref]) +
// (first ? 0 : v[dst]); y = Fermi value.
// Forward encoding (slots reused by liveness): x = dst | first << 6 | leaf << 7 | ref << 8.
constexpr int kOpDstMask = 63, kOpFirst = 1 << 6, kOpLeaf = 1 << 7, kOpRefShift = 8;
constexpr int kMaxSlots = 64;
// Adjoint encoding (one slot per node, ids per diagram): x = dst | first << 20 | leaf << 21 |
// run << 22, y = fv | ref << 12.  run (8 bits) is set on the last leaf edge of a node: its number
// of leaf edges, which share the node's adjoint.
constexpr int kOpbDstBits = 20, kOpbDstMask = (1 << kOpbDstBits) - 1, kOpbFirst = 1 << 20, kOpbLeaf = 1 << 21,
              kOpbRunShift = 22, kOpbFvMask = (1 << 12) - 1, kOpbRefShift = 12, kOpbMaxRef = (1 << 19) - 1;

void set_error(const std::string& msg);

// beta must be finite and positive (the kernels evaluate e^{-beta |x|}); sets the error text.
inline bool beta_ok(double beta) {
  if (beta > 0.0 && std::isfinite(beta)) return true;
  set_error("beta must be finite and positive");
  return false;
}

// Linear form  sum_l i a[l] nu_l + sum_j e[j] E_j.
struct Form {
  std::array<int8_t, kMaxLines> e{};
  std::array<int8_t, kMaxVars> a{};
  bool operator==(const Form& o) const { return e == o.e && a == o.a; }
  bool operator<(const Form& o) const { return e != o.e ? e < o.e : a < o.a; }
};

// d^k/dx^k g_sigma(x) at x = c.E, with g_sigma(x) = 1/(sigma e^{beta x} + 1).
struct FermiFactor {
  std::array<int8_t, kMaxLines> c{};
  int8_t sigma = 1;
  int8_t k = 0;
};

struct SymTerm {
  double A = 1.0;
  std::vector<FermiFactor> F;
  std::vector<std::pair<Form, int>> G;  // distinct Green's functions and their powers
};

// Flattened table.  All offsets are byte offsets into one blob, 16-byte aligned, so the blob
// can be moved into shared memory with bulk copies.  Integer records are int32.  The two
// pole-DAG programs are the last sections, [off_ops, off_opsb) and [off_opsb, bytes), everything
// else lies in [0, off_ops): a forward kernel stages [0, off_opsb), an adjoint kernel [0, off_ops)
// and [off_opsb, bytes), and a forward whose program does not fit beside its tiles stages
// [0, off_ops) and streams the program in chunks.
struct TableHeader {
  int N, nv, m;
  int n_rep;        // lines whose energy is computed (first line of each momentum label)
  int n_rep_ext;    // the first n_rep_ext of them carry the external momentum
  int n_combo, combo_nnz;
  int n_fseg, n_fseg_bose, n_fv;   // Fermi segments (Bose-type first) and values
  int n_lm;                         // nonzero momentum labels of the representative lines
  int n_rden, n_cden;
  int n_g1, n_ops, n_leaves, n_g1rd;
  int max_depth, n_inner;      // pole-tree depth (= m) and inner (non-leaf) edges over all groups
  int n_slots, n_nodes;        // forward value slots (most live in one group); DAG nodes over all groups
  int n_g2, n_g2cd;
  int n_pnode;      // phase-2 product nodes
  int g2_const;     // 1 if group 0 of phase 2 has no frequency-dependent factor (R = 1)
  int max_der;
  int n_ext;        // external frequencies per frequency row (the last n_ext variables)
  int n_xk;         // distinct external-coefficient vectors v_k of the complex denominators
  int bytes;
  // offsets
  int off_alpha;      // double [N][nv]
  int off_repl;       // int32 [n_rep]            rep lines
  int off_lm_ptr;     // int32 [n_rep+1]         nonzero labels per rep line (CSR)
  int off_lm_l;       // int32 [n_lm]             variable index, ascending
  int off_lm_c;       // double [n_lm]            label
  int off_rep_aext;   // double [n_rep]           external label of each rep line
  int off_combo_ptr;  // int32 [n_combo+1]
  int off_combo_j;    // int32 [combo_nnz]        base-energy index, ascending per combo
  int off_combo_c;    // double [combo_nnz]       coefficient
  int off_fseg;       // int32 [n_fseg][8]       combo, sigma, v_begin, first v with k >= 1, v_end
  int off_fv;         // int32 [n_fv][2]         sign, k
  int off_rden;       // int32 [n_rden][2]       combo, sign
  int off_cden;       // int32 [n_cden][2]       combo, sign
  int off_cden_a;     // double [n_cden]          g_c: the external coefficients are g_c * v_{k_c}
  int off_cden_xk;    // int32 [n_cden]           k_c (n_ext = 1: 0, with v_0 = (1) and g_c = a_ext)
  int off_xvec;       // double [n_xk][n_ext]     v_k; the kernels form Y_kf = sum_q v_kq X_fq per row f
  int off_g1;         // int32 [n_g1][4]         op_begin, op_end, rd_begin, rd_end
  int off_g1_tgt;     // int32 [n_g1]             frequency group it feeds (ascending)
  int off_g1_node;    // int32 [n_g1+1]           first adjoint node id of each group (its root)
  int off_leafA;      // double [n_leaves]        merged coefficients of the leaves
  int off_g1rd;       // int32 [n_g1rd][2]       real-den index, power
  int off_g2;         // int32 [n_g2+1]          complex-den offsets
  int off_g2cd;       // int32 [n_g2cd][2]       complex-den index, power
  int off_g2cd_p;     // double [n_g2cd]          the same powers as doubles
  int off_pnode;      // int32 [n_pnode][2]      product node k: value[n_cden+k] = value[src] * value[c]
  int off_g2node;     // int32 [n_g2]             value index of each group's product (-1: R = 1)
  int off_ops;        // int2 [n_ops]            pole-tree program, forward encoding (kOp*)
  int off_opsb;       // int2 [n_ops]            the same program, adjoint encoding (kOpb*)
};

}  // namespace tami

struct tami_diagram {
  int N = 0, nv = 0;
  int n_ext = 1;                      // external variables (the last n_ext of the nv)
  std::vector<int8_t> alpha;          // [N][nv]
  std::vector<uint8_t> boson;         // [nv]
  double prefactor = 1.0;
  std::vector<tami::SymTerm> terms;   // the symbolic solution, released once flattened into blob
  tami_info info{};
  tami::TableHeader hdr{};
  std::vector<unsigned char> blob;    // host copy of the table
  void* d_blob = nullptr;             // device copy
  int device = -1;
  void* jit = nullptr;                // specialised fused kernel of this table (tami_jit.cpp), or null
};

namespace tami {
int flatten(tami_diagram* d);  // terms -> hdr + blob + info
// Specialised kernels (tami_jit.cpp), one per kind of evaluating call.  jit_select: 1 = launch the
// specialised kernel for this call (compiled and cached), 0 = the generic kernel, negative =
// -status (the "always" mode when it cannot be built).  jit_launch writes the generic kernel's
// per-block partial layout for that call into `partial` (at most max_grid rows).
enum { kJitKindFused = 0, kJitKindFwd = 1, kJitKindBwd = 2, kJitKindEnergy = 3 };
// generic_ok = false: the generic kernel cannot take the table (auto mode then specialises at any size)
int jit_select(tami_diagram* d, int kind, int64_t n, int n_f, bool generic_ok = true);
// How the generic forward kernels stage a table (tami_set_table_staging): TAMI_STAGING_AUTO keeps
// the pole-DAG program resident when it fits beside the tiles, TAMI_STAGING_STREAMED always
// streams it through the ring in chunks of ring_chunk_ops() ops.
int staging_mode();
int ring_chunk_ops();
// Bound of the first stage of every mbarrier wait of the generic kernels (tami_debug_set_wait_limit).
long long wait_limit();
int jit_launch(tami_diagram* d, int kind, const tami_lattice* lat, uint64_t seed, uint64_t offset, int64_t n,
               const double* X, int n_f, double beta, const double* gout, double* per_sample, double* ps_dX,
               double* ps_grad, double* saved, double* partial, int max_grid, struct CUstream_st* st, int* grid_out);
// A compiled specialised kernel held apart from its diagram (a batch keeps its diagrams' kernels
// loaded after the diagrams are gone).  jit_handle compiles if needed; jit_grid sets the shared
// memory attribute and returns the launch's grid (resident blocks, capped by the tiles and
// max_grid); jit_launch_at only launches (legal inside a stream capture).  With params non-NULL the
// kernel reads (t, t', mu, kx, ky, beta) from that device array instead of lat and beta.
struct JitHandle {
  std::shared_ptr<void> lib;
  void* fn = nullptr;
  int block = 128;     // threads per block
  size_t smem = 0;
};
int jit_handle(tami_diagram* d, int kind, int n_f, JitHandle* h);
int jit_grid(const JitHandle& h, int64_t n, int max_grid, int* grid);
int jit_launch_at(const JitHandle& h, int grid, const tami_lattice* lat, const double* params, uint64_t seed,
                  uint64_t offset, int64_t n, const double* X, int n_f, double beta, const double* gout,
                  double* per_sample, double* ps_dX, double* ps_grad, double* saved, double* partial,
                  struct CUstream_st* st);
// Disk cache of compiled specialised kernels.  An entry holds the identity of its compilation
// (compiler version, options, device arithmetic, kernel source), the cubin and a checksum of both;
// jit_cache_read accepts an entry only when the file is whole, its identity equals `ident` byte for
// byte and the checksum matches, so a damaged or foreign entry never reaches the driver.
// jit_cache_write writes a temporary file and renames it over `path`.
uint64_t jit_fnv1a(const void* p, size_t n, uint64_t h = 1469598103934665603ull);
bool jit_cache_read(const std::string& path, const std::string& ident, std::vector<char>* cubin);
bool jit_cache_write(const std::string& path, const std::string& ident, const std::vector<char>& cubin);
// Which diagrams of a batch take their specialised forward kernel (use[d] = 1; compiled here on
// parallel host threads): none in mode "never"; in "auto" those with >= 2^20 samples whose kernel
// builds; in "always" every diagram, else the status of the first that cannot be built.
int jit_select_batch(tami_diagram* const* ds, int n_d, const int64_t* n, int n_f, int* use);
void jit_mark_generic(tami_diagram* d);
void jit_release(tami_diagram* d);
// Runs an entry point's body and turns a C++ exception (host memory exhausted, a thread that could
// not be started) into a status with a message: nothing throws across the C ABI.
template <class F>
int guarded(F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    set_error("out of host memory");
    return TAMI_ENOMEM;
  } catch (const std::exception& e) {
    set_error(std::string("host error: ") + e.what());
    return TAMI_EINVAL;
  } catch (...) {
    set_error("host error");
    return TAMI_EINVAL;
  }
}
// Distinct prefixes of the pole DAG's fma chains (tami_host.cpp).  A node's value is a chain
// val = fma(F_y, operand, val) from 0 over its ops in program order; chains of different nodes that
// begin with the same steps share those partial sums, and so do chains that are the same steps with
// every sign flipped: a prefix stands for a partial sum up to its sign (op_sign, node_sign), since
// fma(F, -a, -c) = -fma(F, a, c) exactly in round-to-nearest (a chain's first product onto +0.0 may
// differ in the sign of a zero result only).  A prefix's value is fma(F_fv, osign * operand,
// parent's value), the sign of a node operand's own prefix folded into osign.  An operand that is
// identically zero (a leaf coefficient 0: terms that cancelled exactly when merged; a node made only
// of such) adds nothing and creates no prefix.  Every prefix is
// created by the first op that reaches it, so prefixes come in program order and a node's value is
// complete before any prefix references it.  Input: the adjoint encoding's ops (pairs {x, y}, kOpb*
// fields) and the leaf coefficients (leaves with equal coefficients are the same operand).
struct DagPrefix {
  int parent;    // prefix this one extends, -1 for a chain's first step
  int fv;        // Fermi value F_y
  int node;      // 0: operand is leaf coefficient osign * leafA[operand]; 1: osign * the value (prefix) `operand`
  int operand;
  int osign;     // +1 or -1
};
struct DagPrefixes {
  std::vector<DagPrefix> p;        // creation order
  std::vector<int> op_prefix;      // op -> the prefix it lands on (-1: the partial sum is still zero)
  std::vector<signed char> op_sign;    // op's partial sum = op_sign * that prefix's value
  std::vector<char> op_new;        // op creates that prefix
  std::vector<int> node_value;     // node id -> prefix holding its value (-1: identically zero)
  std::vector<signed char> node_sign;  // node's value = node_sign * that prefix's value
};
DagPrefixes dag_prefixes(const int* opsb, int n_ops, const double* leafA);
// Checks every index and range of a flattened table (tami_validate.cpp); false with the reason.
bool validate_table(const TableHeader& h, const unsigned char* blob, size_t size, std::string* why);
}
