// Many diagrams of uneven order and term count, times many external frequencies, in one
// persistent launch (no counterpart in the paper, which evaluates one diagram per call).
//
// Plan (host, once): every diagram's table is packed into one device buffer; its sample stream is
// cut into work items of `chunk` tiles of 128 samples; the items are sorted by estimated cost,
// largest first (longest-processing-time order); the launch -- reset of the queue counter, the
// persistent kernel and the reduction kernel -- is captured once into a CUDA graph.
// Launch: blocks pop items from an atomic counter; a block restages the table in shared memory
// (bulk copy on an mbarrier) only when the next item belongs to another diagram; it runs the
// forward tiles of the item and stores the item's block-reduced partial sums.  The reduction
// kernel sums each diagram's items in tile order, so results do not depend on which block ran
// which item.  The chunk size and the grid come from a small autotuner (timed graph replays),
// cached per GPU and batch signature in memory and in a text file.
// Specialised diagrams: a diagram whose own generated forward kernel is taken (mode "always", or
// "auto" at >= 2^20 samples) is not cut into items; the graph launches that kernel over the
// diagram's whole sample stream after the persistent kernel, reading the launch's parameters
// from the batch's device buffer, and its per-block partial sums join the diagram's list for the
// same reduction (summed in block order).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <sys/stat.h>

#include "tami_device.cuh"
#include "tami_fwd_tile.cuh"
#include "tami_internal.h"

namespace tami {
namespace {

using namespace dev;

struct BatchDiag {
  TableHeader h;
  long long blob_off;
  unsigned long long seed;
  long long n;
  long long tiles;
};

struct BatchItem {
  int d;
  int pad;
  long long tile0, tile1;
};

struct BatchParams {
  const BatchDiag* diags;
  int n_d;
  const BatchItem* items;
  int n_items;
  const unsigned char* blobs;
  const double* params;   // t, t', mu, kx, ky, beta
  const double* X;
  int n_f;
  int table_cap, max_cden, max_g2;   // largest staged table part (bytes), denominators and groups
  int ring_chunk;         // streamed programs: ops per ring buffer; 0 when every program is resident
  long long wait_limit;   // bound of the first stage of every mbarrier wait
  int* counter;
  int* status;
  double* partial;        // [n_items][n_f][4]
};

// Shared memory: staged table part (table_cap: [0, off_opsb) of the largest table, or [0, off_ops)
// with streamed programs) | ring [2][ring_chunk] ops | Xs | AXI, AXI2 | CB | W | red
size_t batch_smem_bytes(int table_cap, int ring_chunk, int n_f, int max_cden, int max_g2) {
  return (size_t)table_cap + 2 * 8 * (size_t)ring_chunk +
         sizeof(double) * ((2 + 2 * (size_t)max_cden) * n_f + (size_t)(max_cden + max_g2 + 4) * kBlock);
}

template <bool STREAM>
__global__ void __launch_bounds__(kBlock) batch_kernel(const BatchParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ TableHeader Hs;
  __shared__ __align__(8) unsigned long long bar;
  __shared__ __align__(8) unsigned long long ring_bar[2];
  __shared__ int s_item;
  const int tid = threadIdx.x;
  const int n_f = P.n_f;
  unsigned char* tab = smem;
  const int ring_chunk = STREAM ? P.ring_chunk : 0;
  double* Xs = reinterpret_cast<double*>(smem + P.table_cap + 2 * 8 * (size_t)ring_chunk);
  double* AXI = Xs + 2 * n_f;
  double* AXI2 = AXI + P.max_cden * n_f;
  double* CB = AXI2 + P.max_cden * n_f;
  double* W = CB + P.max_cden * kBlock;
  double* red = W + P.max_g2 * kBlock;
  for (int i = tid; i < 2 * n_f; i += kBlock) Xs[i] = P.X[i];
  mbar_init(&bar);
  OpRing R;
  if (STREAM) {
    mbar_init(&ring_bar[0]);
    mbar_init(&ring_bar[1]);
    R.buf = reinterpret_cast<int2*>(smem + P.table_cap);
    R.bar = ring_bar;
    R.status = P.status;
    R.limit = P.wait_limit;
    R.chunk = ring_chunk;
    R.waits[0] = R.waits[1] = 0;
    R.failed = false;
  }
  const FreqMap M = freq_map(n_f, tid);
  TileArgs A;
  A.t = P.params[0]; A.tp = P.params[1]; A.mu = P.params[2]; A.kx = P.params[3]; A.ky = P.params[4];
  A.beta = P.params[5];
  A.offset = 0;
  A.E_in = nullptr;
  A.per_sample = nullptr;
  A.saved = nullptr;
  A.n_f = n_f;
  int cur_d = -1;
  uint32_t phase = 0;
  bool xr_zero = true;
  double acc[kMaxFreqPerThread][4];
  __syncthreads();
  while (true) {
    if (tid == 0) s_item = atomicAdd(P.counter, 1);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= P.n_items) break;
    const BatchItem item = P.items[it];
    const int d = item.d;
    if (d < 0 || d >= P.n_d || item.tile0 < 0 || item.tile1 > P.diags[d].tiles || item.tile0 >= item.tile1) {
      if (tid == 0) atomicExch(P.status, TAMI_EINVAL);   // malformed queue entry: skip it
      continue;
    }
    if (d != cur_d) {
      if (tid == 0) Hs = P.diags[d].h;
      __syncthreads();
      const bool ok = bulk_stage(tab, P.blobs + P.diags[d].blob_off, STREAM ? Hs.off_ops : Hs.off_opsb, &bar, phase,
                                 P.status, P.wait_limit);
      if (__syncthreads_or(!ok)) return;
      phase ^= 1u;
      cur_d = d;
      if (STREAM) {
        R.src = P.blobs + P.diags[d].blob_off + Hs.off_ops;
        R.n_ops = Hs.n_ops;
        R.n_chunks = (Hs.n_ops + ring_chunk - 1) / ring_chunk;
      }
      xr_zero = freq_constants(Hs, table_view(tab, Hs), Xs, n_f, AXI, AXI2);
    }
    const TableView T = table_view(tab, Hs);
    A.seed = P.diags[d].seed;
    A.n = P.diags[d].n;
    for (int i = 0; i < kMaxFreqPerThread; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0;
    for (long long tile = item.tile0; tile < item.tile1; ++tile)
      fwd_tile<false, false, STREAM>(Hs, T, A, tile, Xs, AXI, AXI2, xr_zero, CB, W, M, acc, R);
    block_reduce_store(M, n_f, acc, red, P.partial + (size_t)it * n_f * 4);
  }
}

// mean and variance of every (diagram, frequency) from its items, summed in tile order
__global__ void batch_reduce_kernel(const double* partial, const int* item_ptr, const int* item_list,
                                    const BatchDiag* diags, int n_d, int n_f, const int* status, double* mean,
                                    double* var) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_d * n_f) return;
  const int d = i / n_f, f = i % n_f;
  double s1r = 0.0, s1i = 0.0, s2r = 0.0, s2i = 0.0;
  for (int q = item_ptr[d]; q < item_ptr[d + 1]; ++q) {
    const double* p = partial + ((size_t)item_list[q] * n_f + f) * 4;
    s1r += p[0]; s1i += p[1]; s2r += p[2]; s2i += p[3];
  }
  const long long n = diags[d].n;
  const double nn = (double)n;
  double mr = s1r / nn, mi = s1i / nn;
  double vr = n > 1 ? (s2r - s1r * mr) / (nn - 1.0) : 0.0;
  double vi = n > 1 ? (s2i - s1i * mi) / (nn - 1.0) : 0.0;
  if (*status != 0) mr = mi = vr = vi = __longlong_as_double(0x7ff8000000000000ll);
  mean[2 * i] = mr;
  mean[2 * i + 1] = mi;
  var[2 * i] = vr;
  var[2 * i + 1] = vi;
}

// ------------------------------------------------------------------------------ host side
size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

struct Layout {
  size_t diags, items, item_ptr, item_list, blobs, params, X, ctr, partial, mean, var, total;
};

}  // namespace
}  // namespace tami

using namespace tami;

struct tami_batch {
  int device = -1;
  int n_d = 0, n_f = 0;
  std::vector<const tami_diagram*> ds;
  std::vector<int64_t> n;
  std::vector<uint64_t> seeds;
  int chunk = 0, grid = 0, n_items = 0;
  int table_cap = 0, max_cden = 0, max_g2 = 0;   // over the diagrams the persistent kernel runs
  int ring_chunk = 0;                              // streamed programs: ops per ring buffer
  std::vector<int> spec;                           // 1: the diagram runs its specialised kernel
  std::vector<tami::JitHandle> jit;                // those kernels, kept loaded by the batch
  std::vector<int> jit_grid;
  int n_spec = 0;
  size_t smem = 0;
  Layout L{};
  unsigned char* mem = nullptr;
  cudaStream_t cap = nullptr;
  // the specialised launches go to parallel branches of the graph (forked from and joined back to
  // cap), so that one launch's blocks fill the SMs another launch's tail leaves idle
  static constexpr int kBranches = 4;
  cudaStream_t br[kBranches] = {};
  cudaEvent_t ev_fork = nullptr, ev_join[kBranches] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double tuned_ms = -1.0;
};

namespace tami {
namespace {

void release_graph(tami_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->mem) cudaFree(b->mem);
  b->exec = nullptr;
  b->graph = nullptr;
  b->mem = nullptr;
}

void release_streams(tami_batch* b) {
  for (int i = 0; i < tami_batch::kBranches; ++i) {
    if (b->br[i]) cudaStreamDestroy(b->br[i]);
    if (b->ev_join[i]) cudaEventDestroy(b->ev_join[i]);
    b->br[i] = nullptr;
    b->ev_join[i] = nullptr;
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  b->ev_fork = nullptr;
  b->cap = nullptr;
}

// Build items, device buffers and the graph for one (chunk, grid) choice; with_spec = false
// leaves the specialised diagrams out (tuning replays time the persistent kernel alone).
int build(tami_batch* b, int chunk, int grid_cap, bool with_spec) {
  release_graph(b);
  const int n_d = b->n_d, n_f = b->n_f;
  std::vector<BatchDiag> diags(n_d);
  std::vector<double> cost_per_tile(n_d);
  size_t blob_bytes = 0;
  for (int d = 0; d < n_d; ++d) {
    const tami_diagram* D = b->ds[d];
    diags[d].h = D->hdr;
    diags[d].blob_off = (long long)blob_bytes;
    blob_bytes += up256(D->blob.size());
    diags[d].seed = b->seeds[d];
    diags[d].n = b->n[d];
    diags[d].tiles = (b->n[d] + kBlock - 1) / kBlock;
    cost_per_tile[d] = kBlock * (D->info.flops_per_sample + n_f * D->info.flops_per_sample_freq);
  }
  std::vector<BatchItem> items;
  for (int d = 0; d < n_d; ++d)
    for (long long t = 0; !b->spec[d] && t < diags[d].tiles; t += chunk)
      items.push_back({d, 0, t, std::min<long long>(t + chunk, diags[d].tiles)});
  std::stable_sort(items.begin(), items.end(), [&](const BatchItem& x, const BatchItem& y) {
    return (x.tile1 - x.tile0) * cost_per_tile[x.d] > (y.tile1 - y.tile0) * cost_per_tile[y.d];
  });
  const int n_items = (int)items.size();
  // partial rows: the items', then each specialised launch's blocks
  std::vector<long long> spec_row(n_d, -1);
  long long n_rows = n_items;
  for (int d = 0; d < n_d; ++d)
    if (with_spec && b->spec[d]) { spec_row[d] = n_rows; n_rows += b->jit_grid[d]; }
  std::vector<int> item_ptr(n_d + 1, 0), item_list((size_t)n_rows);
  {
    std::vector<std::vector<std::pair<long long, int>>> per(n_d);
    for (int i = 0; i < n_items; ++i) per[items[i].d].push_back({items[i].tile0, i});
    int q = 0;
    for (int d = 0; d < n_d; ++d) {
      std::sort(per[d].begin(), per[d].end());
      item_ptr[d] = q;
      for (auto& pr : per[d]) item_list[q++] = pr.second;
      if (spec_row[d] >= 0)
        for (int r = 0; r < b->jit_grid[d]; ++r) item_list[q++] = (int)(spec_row[d] + r);
    }
    item_ptr[n_d] = q;
  }
  Layout& L = b->L;
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off += up256(bytes); return o; };
  L.diags = take(sizeof(BatchDiag) * n_d);
  L.items = take(sizeof(BatchItem) * n_items);
  L.item_ptr = take(sizeof(int) * (n_d + 1));
  L.item_list = take(sizeof(int) * n_rows);
  L.blobs = take(blob_bytes);
  L.params = take(sizeof(double) * 8);
  L.X = take(sizeof(double) * 2 * n_f);
  L.ctr = take(256);
  L.partial = take(sizeof(double) * 4 * (size_t)n_f * n_rows);
  L.mean = take(sizeof(double) * 2 * (size_t)n_f * n_d);
  L.var = take(sizeof(double) * 2 * (size_t)n_f * n_d);
  L.total = off;
  cudaError_t e = cudaMalloc(&b->mem, L.total);
  if (e != cudaSuccess) { b->mem = nullptr; set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e)); return TAMI_ENOMEM; }
  std::vector<unsigned char> host(L.blobs + blob_bytes, 0);
  std::memcpy(host.data() + L.diags, diags.data(), sizeof(BatchDiag) * n_d);
  std::memcpy(host.data() + L.items, items.data(), sizeof(BatchItem) * n_items);
  std::memcpy(host.data() + L.item_ptr, item_ptr.data(), sizeof(int) * (n_d + 1));
  std::memcpy(host.data() + L.item_list, item_list.data(), sizeof(int) * n_rows);
  for (int d = 0; d < n_d; ++d)
    std::memcpy(host.data() + L.blobs + diags[d].blob_off, b->ds[d]->blob.data(), b->ds[d]->blob.size());
  e = cudaMemcpy(b->mem, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy");
  e = cudaMemset(b->mem + L.params, 0, L.partial - L.params);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemset");
  // grid: resident blocks, capped
  DeviceProps dp = device_props(b->device);
  b->smem = batch_smem_bytes(b->table_cap, b->ring_chunk, n_f, b->max_cden, b->max_g2);
  if (b->smem > dp.smem_optin) {
    set_error("largest table and tiles exceed shared memory even with the pole-DAG programs streamed");
    return TAMI_EUNSUPPORTED;
  }
  const void* kfn = b->ring_chunk ? (const void*)batch_kernel<true> : (const void*)batch_kernel<false>;
  e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem);
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kBlock, b->smem);
  if (e != cudaSuccess) return cuda_fail(e, "occupancy");
  int grid = std::max(1, dp.sms * std::max(per_sm, 1));
  if (grid_cap > 0) grid = std::min(grid, grid_cap);
  grid = std::min(grid, n_items);   // 0: every diagram is specialised
  b->grid = grid;
  b->chunk = chunk;
  b->n_items = n_items;
  // graph: reset counter/status, persistent kernel, reduction
  BatchParams P;
  std::memset(&P, 0, sizeof(P));
  P.diags = reinterpret_cast<const BatchDiag*>(b->mem + L.diags);
  P.n_d = n_d;
  P.items = reinterpret_cast<const BatchItem*>(b->mem + L.items);
  P.n_items = n_items;
  P.blobs = b->mem + L.blobs;
  P.params = reinterpret_cast<const double*>(b->mem + L.params);
  P.X = reinterpret_cast<const double*>(b->mem + L.X);
  P.n_f = n_f;
  P.table_cap = b->table_cap;
  P.ring_chunk = b->ring_chunk;
  P.wait_limit = wait_limit();
  P.max_cden = b->max_cden;
  P.max_g2 = b->max_g2;
  P.counter = reinterpret_cast<int*>(b->mem + L.ctr);
  P.status = reinterpret_cast<int*>(b->mem + L.ctr) + 1;
  P.partial = reinterpret_cast<double*>(b->mem + L.partial);
  e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
  cudaMemsetAsync(b->mem + L.ctr, 0, 2 * sizeof(int), b->cap);
  int n_br = 0;
  for (int d = 0; d < n_d; ++d) if (spec_row[d] >= 0) ++n_br;
  if (n_br > tami_batch::kBranches) n_br = tami_batch::kBranches;
  if (n_br > 0) {
    cudaEventRecord(b->ev_fork, b->cap);
    for (int i = 0; i < n_br; ++i) cudaStreamWaitEvent(b->br[i], b->ev_fork, 0);
  }
  if (n_items > 0) {
    if (b->ring_chunk) batch_kernel<true><<<grid, kBlock, b->smem, b->cap>>>(P);
    else batch_kernel<false><<<grid, kBlock, b->smem, b->cap>>>(P);
  }
  int rc = TAMI_OK;
  for (int d = 0, k = 0; d < n_d && rc == TAMI_OK; ++d)
    if (spec_row[d] >= 0)
      rc = jit_launch_at(b->jit[d], b->jit_grid[d], nullptr, P.params, b->seeds[d], 0, b->n[d], P.X, n_f, 0.0,
                         nullptr, nullptr, nullptr, nullptr, nullptr, P.partial + (size_t)spec_row[d] * n_f * 4,
                         b->br[k++ % n_br]);
  for (int i = 0; i < n_br; ++i) {
    cudaEventRecord(b->ev_join[i], b->br[i]);
    cudaStreamWaitEvent(b->cap, b->ev_join[i], 0);
  }
  const int nt = n_d * n_f;
  batch_reduce_kernel<<<(nt + 127) / 128, 128, 0, b->cap>>>(
      P.partial, reinterpret_cast<const int*>(b->mem + L.item_ptr), reinterpret_cast<const int*>(b->mem + L.item_list),
      P.diags, n_d, n_f, P.status, reinterpret_cast<double*>(b->mem + L.mean), reinterpret_cast<double*>(b->mem + L.var));
  e = cudaStreamEndCapture(b->cap, &b->graph);
  if (rc) return rc;
  if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
  return TAMI_OK;
}

// Autotune cache: key -> (chunk, grid), in memory and in a text file.
std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune;

std::string tune_path() {
  const char* p = std::getenv("TAMI_TUNE_CACHE");
  if (p && *p) return p;
  const char* h = std::getenv("HOME");
  return std::string(h ? h : ".") + "/.cache/libtami_autotune.txt";
}

std::string tune_key(const tami_batch* b) {
  cudaDeviceProp p;
  cudaGetDeviceProperties(&p, b->device);
  unsigned long long hsh = 1469598103934665603ull;
  auto mix = [&](unsigned long long v) { hsh = (hsh ^ v) * 1099511628211ull; };
  for (int d = 0; d < b->n_d; ++d) {
    if (b->spec[d]) continue;   // not run by the tuned kernel
    mix((unsigned long long)b->ds[d]->info.n_terms);
    mix((unsigned long long)b->n[d]);
    mix((unsigned long long)b->ds[d]->blob.size());
  }
  char buf[512];
  std::snprintf(buf, sizeof(buf), "%s|sm%d|nd%d|nf%d|%016llx", p.name, p.multiProcessorCount, b->n_d - b->n_spec,
                b->n_f, hsh);
  std::string k(buf);
  for (char& c : k) if (c == ' ' || c == '\t') c = '_';
  return k;
}

bool tune_lookup(const std::string& key, int* chunk, int* grid) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(key);
  if (it == g_tune.end()) {
    FILE* f = std::fopen(tune_path().c_str(), "r");
    if (f) {
      char k[512];
      int c, g;
      while (std::fscanf(f, "%511s %d %d", k, &c, &g) == 3) g_tune[k] = {c, g};
      std::fclose(f);
    }
    it = g_tune.find(key);
  }
  if (it == g_tune.end()) return false;
  *chunk = it->second.first;
  *grid = it->second.second;
  return true;
}

void tune_store(const std::string& key, int chunk, int grid) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = {chunk, grid};
  std::string path = tune_path();
  const size_t slash = path.find_last_of('/');
  if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);   // may exist
  FILE* f = std::fopen(path.c_str(), "a");
  if (f) {
    std::fprintf(f, "%s %d %d\n", key.c_str(), chunk, grid);
    std::fclose(f);
  }
}

// Typical inputs for tuning replays: t = 1, mu = 0, k_ext = (pi/2, pi/2), beta = 5, i(2f+1)pi/beta.
void tuning_inputs(tami_batch* b) {
  const double beta = 5.0, pi = 3.141592653589793;
  const double params[6] = {1.0, 0.0, 0.0, pi / 2, pi / 2, beta};
  std::vector<double> X(2 * b->n_f);
  for (int f = 0; f < b->n_f; ++f) { X[2 * f] = 0.0; X[2 * f + 1] = (2 * f + 1) * pi / beta; }
  cudaMemcpy(b->mem + b->L.params, params, sizeof(params), cudaMemcpyHostToDevice);
  cudaMemcpy(b->mem + b->L.X, X.data(), sizeof(double) * X.size(), cudaMemcpyHostToDevice);
}

// Each timed candidate of a tuning run is appended to $TAMI_TUNE_LOG, when it is set, as one line
// "<plan key> chunk=<tiles per item> grid=<blocks> items=<n> ms=<per replay>", for sweep records.
void tune_log(const std::string& key, const tami_batch* b, double ms) {
  const char* p = std::getenv("TAMI_TUNE_LOG");
  if (!p || !*p) return;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  if (FILE* f = std::fopen(p, "a")) {
    std::fprintf(f, "%s chunk=%d grid=%d items=%d ms=%.4f\n", key.c_str(), b->chunk, b->grid, b->n_items, ms);
    std::fclose(f);
  }
}

double time_replays(tami_batch* b, int reps) {
  tuning_inputs(b);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaGraphLaunch(b->exec, b->cap);   // warm-up
  cudaEventRecord(e0, b->cap);
  for (int r = 0; r < reps; ++r) cudaGraphLaunch(b->exec, b->cap);
  cudaEventRecord(e1, b->cap);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms / reps;
}

}  // namespace
}  // namespace tami

extern "C" {

int tami_batch_plan(const tami_diagram* const* ds, int n_d, const int64_t* samples, const uint64_t* seeds, int n_f,
                    int chunk_tiles, tami_batch** out) {
  return guarded([&]() -> int {
  if (!ds || !samples || !seeds || !out || n_d < 1 || n_f < 1 || n_f > kMaxFreqPerThread * kBlock) {
    set_error("bad argument (n_d >= 1, 1 <= n_f <= 2048, non-NULL arrays)");
    return TAMI_EINVAL;
  }
  *out = nullptr;
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  tami_batch* b = new (std::nothrow) tami_batch;
  if (!b) { set_error("out of host memory"); return TAMI_ENOMEM; }
  b->device = dev;
  b->n_d = n_d;
  b->n_f = n_f;
  for (int d = 0; d < n_d; ++d) {
    if (!ds[d] || samples[d] < 1) { delete b; set_error("NULL diagram or empty sample count"); return TAMI_EINVAL; }
    if (ds[d]->n_ext != 1) {
      delete b;
      set_error("momentum sampling takes one external frequency and momentum (n_ext = 1)");
      return TAMI_EUNSUPPORTED;
    }
    b->ds.push_back(ds[d]);
    b->n.push_back(samples[d]);
    b->seeds.push_back(seeds[d]);
  }
  // specialised diagrams (compiled now); the kernel cache is state of the diagram object, not of
  // the table the batch copies
  b->spec.assign(n_d, 0);
  b->jit.resize(n_d);
  b->jit_grid.assign(n_d, 0);
  {
    std::vector<tami_diagram*> mut(n_d);
    for (int d = 0; d < n_d; ++d) mut[d] = const_cast<tami_diagram*>(ds[d]);
    int rc = jit_select_batch(mut.data(), n_d, samples, n_f, b->spec.data());
    for (int d = 0; d < n_d && rc == TAMI_OK; ++d) {
      if (!b->spec[d]) continue;
      rc = jit_handle(mut[d], kJitKindFwd, n_f, &b->jit[d]);
      if (!rc) rc = jit_grid(b->jit[d], samples[d], 1 << 30, &b->jit_grid[d]);
      ++b->n_spec;
    }
    if (rc) { delete b; return rc; }
  }
  // staging: every forward program resident beside the tiles when the largest fits (and streaming
  // is not forced), else the programs streamed through the ring
  int cap_res = 0, cap_prog = 0;
  for (int d = 0; d < n_d; ++d) {
    if (b->spec[d]) continue;
    cap_res = std::max(cap_res, ds[d]->hdr.off_opsb);
    cap_prog = std::max(cap_prog, ds[d]->hdr.off_ops);
    b->max_cden = std::max(b->max_cden, ds[d]->hdr.n_cden);
    b->max_g2 = std::max(b->max_g2, ds[d]->hdr.n_g2);
  }
  {
    const size_t optin = device_props(b->device).smem_optin;
    if (staging_mode() != TAMI_STAGING_STREAMED &&
        batch_smem_bytes(cap_res, 0, n_f, b->max_cden, b->max_g2) <= optin) {
      b->table_cap = cap_res;
      b->ring_chunk = 0;
    } else {
      b->table_cap = cap_prog;
      b->ring_chunk = ring_chunk_ops();
    }
  }
  e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  if (e != cudaSuccess) { delete b; return cuda_fail(e, "cudaStreamCreate"); }
  for (int i = 0; i < tami_batch::kBranches && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->br[i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[i], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  if (e != cudaSuccess) { release_streams(b); delete b; return cuda_fail(e, "cudaStreamCreate"); }
  int rc = TAMI_OK;
  if (chunk_tiles > 0) {
    rc = build(b, chunk_tiles, 0, true);
  } else if (b->n_spec == n_d) {
    rc = build(b, 1, 0, true);   // no items: nothing to tune
  } else {
    const std::string key = tune_key(b);
    int c = 0, g = 0;
    if (tune_lookup(key, &c, &g)) {
      rc = build(b, c, g, true);
    } else {
      // candidates: chunk sizes giving about 2..32 items per resident block, full grid
      long long tiles = 0;
      for (int d = 0; d < n_d; ++d)
        if (!b->spec[d]) tiles += (b->n[d] + kBlock - 1) / kBlock;
      DeviceProps dp = device_props(dev);
      const long long slots = (long long)dp.sms * 8;
      std::vector<int> cands;
      for (int per : {2, 4, 8, 16, 32}) {
        int ch = (int)std::max<long long>(1, tiles / (slots * per));
        if (std::find(cands.begin(), cands.end(), ch) == cands.end()) cands.push_back(ch);
      }
      double best = 1e300;
      int best_c = cands[0], best_g = 0;
      for (int ch : cands) {
        rc = build(b, ch, 0, false);
        if (rc) break;
        double ms = time_replays(b, 2);
        tune_log(key, b, ms);
        if (ms < best) { best = ms; best_c = ch; }
      }
      // then the residency at that work-item size: 1, 2, 4 ... blocks per SM up to the resident
      // maximum the full grid has (fewer resident blocks: more shared memory and L1 per block)
      if (!rc) rc = build(b, best_c, 0, false);
      if (!rc) {
        const int full = b->grid;
        for (int per = 1; per * dp.sms < full && !rc; per *= 2) {
          rc = build(b, best_c, per * dp.sms, false);
          if (rc) break;
          double ms = time_replays(b, 2);
          tune_log(key, b, ms);
          if (ms < best) { best = ms; best_g = per * dp.sms; }
        }
      }
      if (!rc) {
        rc = build(b, best_c, best_g, true);
        b->tuned_ms = best;
        if (!rc) tune_store(key, b->chunk, b->grid);
      }
    }
  }
  if (rc) {
    release_graph(b);
    release_streams(b);
    delete b;
    return rc;
  }
  *out = b;
  return TAMI_OK;
  });
}

int tami_batch_info(const tami_batch* b, int* n_items, int* grid, int* chunk_tiles) {
  if (!b) { set_error("NULL batch"); return TAMI_EINVAL; }
  if (n_items) *n_items = b->n_items;
  if (grid) *grid = b->grid;
  if (chunk_tiles) *chunk_tiles = b->chunk;
  return TAMI_OK;
}

int tami_batch_specialised(const tami_batch* b, int* flags, int* n_specialised) {
  if (!b) { set_error("NULL batch"); return TAMI_EINVAL; }
  if (flags)
    for (int d = 0; d < b->n_d; ++d) flags[d] = b->spec[d];
  if (n_specialised) *n_specialised = b->n_spec;
  return TAMI_OK;
}

int tami_batch_debug_set_item(tami_batch* b, int item, int d, int64_t tile0, int64_t tile1, int64_t* prev) {
  if (!b || !b->mem || item < 0 || item >= b->n_items) { set_error("bad argument"); return TAMI_EINVAL; }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != b->device) { set_error("current device differs from the plan's device"); return TAMI_EINVAL; }
  BatchItem* p = reinterpret_cast<BatchItem*>(b->mem + b->L.items) + item;
  BatchItem old{};
  cudaError_t e = cudaMemcpy(&old, p, sizeof(old), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy item");
  if (prev) { prev[0] = old.d; prev[1] = old.tile0; prev[2] = old.tile1; }
  const BatchItem now{d, 0, tile0, tile1};
  e = cudaMemcpy(p, &now, sizeof(now), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? TAMI_OK : cuda_fail(e, "cudaMemcpy item");
}

int tami_batch_launch(tami_batch* b, const tami_lattice* lat, const double* X, double beta, double* mean, double* var,
                      tami_stream_t stream) {
  if (!b || !lat || !X || !mean) { set_error("bad argument"); return TAMI_EINVAL; }
  if (!beta_ok(beta)) return TAMI_EINVAL;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != b->device) { set_error("current device differs from the plan's device"); return TAMI_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  const double params[6] = {lat->t, lat->tp, lat->mu, lat->kx_ext, lat->ky_ext, beta};
  // pageable source: the copy has consumed `params` when the call returns
  cudaError_t e = cudaMemcpyAsync(b->mem + b->L.params, params, sizeof(params), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync params");
  e = cudaMemcpyAsync(b->mem + b->L.X, X, sizeof(double) * 2 * b->n_f, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync X");
  e = cudaGraphLaunch(b->exec, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
  const size_t out_bytes = sizeof(double) * 2 * (size_t)b->n_f * b->n_d;
  e = cudaMemcpyAsync(mean, b->mem + b->L.mean, out_bytes, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync mean");
  if (var) {
    e = cudaMemcpyAsync(var, b->mem + b->L.var, out_bytes, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpyAsync var");
  }
  return TAMI_OK;
}

void tami_batch_destroy(tami_batch* b) {
  if (!b) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  release_graph(b);
  release_streams(b);
  if (prev >= 0) cudaSetDevice(prev);
  delete b;
}

}  // extern "C"
