// Device side of libtami: evaluation of a flattened AMI term table over Monte Carlo momentum
// samples (Sec. 5.2) or given energies (Sec. 2.3) on sm_103a, FP64/complex128 throughout.
//
// Work split.  One thread block owns a tile of S samples at a time:
//   phase 1 (one thread per sample, frequency independent, Sec. 2.2 "FT is not a function of
//     the external frequencies"): Philox momenta -> line momenta -> energies -> energy
//     combinations -> Fermi/Bose values and their derivatives -> per group of terms sharing
//     one denominator signature, sum_t A_t prod FT factors, times the frequency-independent
//     denominators -> W[group][sample] in shared memory;
//   phase 2 (threads over (frequency, sample) pairs): the frequency-dependent reciprocals
//     1/(a X_f + b) once per denominator, the per-group products, and the sum over groups.
// Sums over samples stay in registers per thread, are reduced per block in a fixed order,
// and a second kernel reduces the per-block partials in a fixed order (deterministic).
//
// The term table of the diagram is moved into shared memory once per block with a bulk
// (TMA) copy, cp.async.bulk, completed on an mbarrier whose wait is bounded.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>

#include "tami_device.cuh"
#include "tami_fwd_tile.cuh"
#include "tami_internal.h"

namespace tami {
namespace {

using namespace dev;

struct FwdParams {
  TableHeader h;
  const unsigned char* table;   // device blob, 16-byte aligned, h.bytes long
  double t, tp, mu, kx, ky;
  unsigned long long seed, offset;
  long long n;
  const double* E_in;           // energy input [n][N] or null
  const double* X;              // [n_f][n_ext][2]
  int n_f;
  double beta;
  double* per_sample;           // [n_f][n][2] or null
  double* saved;                // [n_rep + 2 n_rep_ext][n] for the adjoint, or null (momentum mode)
  double* partial;              // [gridDim][n_f][4] or null
  int* status;                  // device status word or null
  int ring_chunk;               // streamed program: ops per ring buffer (even); 0 when resident
  long long wait_limit;         // bound of the first stage of every mbarrier wait
};


// Staged part of the table: [0, off_opsb) (everything the forward reads), or with a streamed
// program [0, off_ops) and the two ring buffers.
__host__ __device__ __forceinline__ size_t fwd_table_smem(const TableHeader& h, int ring_chunk) {
  return ring_chunk ? (size_t)h.off_ops + 2 * 8 * (size_t)ring_chunk : (size_t)h.off_opsb;
}

// Shared memory: table | Xs [n_xk][n_f][2] | AXI, AXI2 [n_cden][n_f] | CB [n_cden][S] | W [n_g2][S] |
// red [4][S]
__host__ __device__ __forceinline__ size_t fwd_smem_bytes(const TableHeader& h, int n_f, int ring_chunk) {
  return fwd_table_smem(h, ring_chunk) +
         sizeof(double) * ((2 * (size_t)h.n_xk + 2 * (size_t)h.n_cden) * n_f + (size_t)(h.n_cden + h.n_g2 + 4) * kBlock);
}

template <bool ENERGY_IN, bool SAVE, bool STREAM>
__global__ void __launch_bounds__(kBlock) fwd_kernel(const FwdParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ __align__(8) unsigned long long ring_bar[2];
  const TableHeader& H = P.h;
  const int tid = threadIdx.x;
  if (!stage_table(smem, P.table, STREAM ? H.off_ops : H.off_opsb, P.status, P.wait_limit)) return;
  OpRing R;
  if (STREAM) {
    mbar_init(&ring_bar[0]);
    mbar_init(&ring_bar[1]);
    R.src = P.table + H.off_ops;
    R.buf = reinterpret_cast<int2*>(smem + H.off_ops);
    R.bar = ring_bar;
    R.status = P.status;
    R.limit = P.wait_limit;
    R.n_ops = H.n_ops;
    R.chunk = P.ring_chunk;
    R.n_chunks = (H.n_ops + P.ring_chunk - 1) / P.ring_chunk;
    R.waits[0] = R.waits[1] = 0;
    R.failed = false;
  }
  double* Xs = reinterpret_cast<double*>(smem + fwd_table_smem(H, STREAM ? P.ring_chunk : 0));
  double* AXI = Xs + 2 * H.n_xk * P.n_f;
  double* AXI2 = AXI + H.n_cden * P.n_f;
  double* CB = AXI2 + H.n_cden * P.n_f;
  double* W = CB + H.n_cden * kBlock;
  double* red = W + H.n_g2 * kBlock;
  const TableView T = table_view(smem, H);
  stage_freqs(H, T, P.X, P.n_f, Xs);
  const FreqMap M = freq_map(P.n_f, tid);
  double acc[kMaxFreqPerThread][4];
  for (int i = 0; i < kMaxFreqPerThread; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.0;
  __syncthreads();
  const bool xr_zero = freq_constants(H, T, Xs, P.n_f, AXI, AXI2);
  TileArgs A;
  A.t = P.t; A.tp = P.tp; A.mu = P.mu; A.kx = P.kx; A.ky = P.ky; A.beta = P.beta;
  A.seed = P.seed; A.offset = P.offset; A.n = P.n; A.E_in = P.E_in; A.per_sample = P.per_sample;
  A.saved = P.saved;
  A.n_f = P.n_f;
  const long long n_tiles = (P.n + kBlock - 1) / kBlock;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x)
    fwd_tile<ENERGY_IN, SAVE, STREAM>(H, T, A, tile, Xs, AXI, AXI2, xr_zero, CB, W, M, acc, R);
  if (!P.partial) return;
  block_reduce_store(M, P.n_f, acc, red, P.partial + (size_t)blockIdx.x * P.n_f * 4);
}

// mean and unbiased variances from per-block partials, summed in block order
// One block of kFinBlock threads per frequency: the sums over the per-block partials.
__global__ void __launch_bounds__(kFinBlock) finalize_kernel(const double* partial, int n_blocks, int n_f, long long n,
                                                            const int* status, double* mean, double* var) {
  __shared__ double sh[4][kFinBlock];
  const int f = blockIdx.x;
  double s[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < n_blocks; b += kFinBlock) {
    const double* p = partial + ((size_t)b * n_f + f) * 4;
    for (int k = 0; k < 4; ++k) s[k] += p[k];
  }
  fixed_tree_sum<4>(s, sh);
  if (threadIdx.x != 0) return;
  const double s1r = s[0], s1i = s[1], s2r = s[2], s2i = s[3];
  const double nn = (double)n;
  double mr = s1r / nn, mi = s1i / nn;
  double vr = n > 1 ? (s2r - s1r * mr) / (nn - 1.0) : 0.0;
  double vi = n > 1 ? (s2i - s1i * mi) / (nn - 1.0) : 0.0;
  if (status && *status != 0) mr = mi = vr = vi = __longlong_as_double(0x7ff8000000000000ll);
  mean[2 * f] = mr;
  mean[2 * f + 1] = mi;
  if (var) { var[2 * f] = vr; var[2 * f + 1] = vi; }
}

__global__ void exp_selftest_kernel(const double* t, long long n, double* y, double* em, double* y_plain) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double e = 0.0;
  y[i] = exp_neg<true>(t[i], e);
  em[i] = e;
  if (y_plain) y_plain[i] = exp_neg<false>(t[i], e);
}

__global__ void sincos_selftest_kernel(const double* k, long long n, double* s, double* c) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double sv, cv;
  cw_sincos(k[i], sv, cv);
  s[i] = sv;
  c[i] = cv;
  // the cosine-only path of the dispersion gives the same bits
  if (__double_as_longlong(cw_cos(k[i])) != __double_as_longlong(cv)) c[i] = __longlong_as_double(0x7ff8000000000000ll);
}

__global__ void imul_selftest_kernel(const double* a, const double* b, long long n, double* mul) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  mul[i] = imul(a[i], b[i]);
}

__global__ void imul_ftz_selftest_kernel(const double* a, const double* b, long long n, double* mul) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  mul[i] = imul_ftz(a[i], b[i]);
}

// FP64 issue-rate probes: C independent fma recurrences per thread, U steps of each per trip, the
// sums written out so that nothing is dropped; 2 C U trips flops per thread.  How fast the FP64
// unit runs them depends on how the operands sit in the register file, so there are several
// operand patterns and a caller takes the fastest:
//   OWN = false: a_k <- a_k m + c, one multiplier and addend for every chain;
//   OWN = true, ACC = false: a_k <- a_k m_k + c_k, each chain its own multiplier and addend;
//   OWN = true, ACC = true: a_k <- m_k c_k + a_k, the chain in the addend (a running sum).
// m_k = m - 1e-9 k, c_k = c + 1e-9 k, |m_k| < 1: bounded, never subnormal.
template <int C, int U, bool OWN, bool ACC>
__global__ void __launch_bounds__(256) fp64_rate_kernel(long long trips, double m, double c, double* out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double a[C], mm[C], cc[C];
#pragma unroll
  for (int k = 0; k < C; ++k) {
    a[k] = 1e-3 * (double)((t + k) & 1023);
    mm[k] = OWN ? m - 1e-9 * k : m;
    cc[k] = OWN ? c + 1e-9 * k : c;
  }
  for (long long it = 0; it < trips; ++it) {
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int k = 0; k < C; ++k) a[k] = ACC ? fma(mm[k], cc[k], a[k]) : fma(a[k], OWN ? mm[k] : m, OWN ? cc[k] : c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < C; ++k) s += a[k];
  out[t] = s;
}

__global__ void sample_energies_kernel(const FwdParams P, double* E) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P.n) return;
  const TableHeader& H = P.h;
  const double* alpha = reinterpret_cast<const double*>(P.table + H.off_alpha);
  double kx[kMaxVars], ky[kMaxVars];
  const unsigned long long sg = P.offset + (unsigned long long)s;
  for (int l = 0; l < H.m; ++l) {
    uint32_t c[4] = {(uint32_t)sg, (uint32_t)(sg >> 32), (uint32_t)l, 0u};
    philox4x32_10(c, (uint32_t)P.seed, (uint32_t)(P.seed >> 32));
    kx[l] = to_momentum(c[0], c[1]);
    ky[l] = to_momentum(c[2], c[3]);
  }
  kx[H.m] = P.kx;
  ky[H.m] = P.ky;
  for (int j = 0; j < H.N; ++j) {
    double ax = 0.0, ay = 0.0;
    for (int l = 0; l < H.nv; ++l) {
      const double cf = alpha[j * H.nv + l];
      if (cf != 0.0) { ax = fma(cf, kx[l], ax); ay = fma(cf, ky[l], ay); }
    }
    E[s * H.N + j] = line_energy(ax, ay, P.t, P.tp, P.mu);
  }
}

// ------------------------------------------------------------------------------- host glue
// How the generic forward stages a table: the program resident beside the tiles when it fits
// (and streaming is not forced), else streamed through the ring; ring_chunk = 0 means resident.
// Returns false when even the streamed layout exceeds shared memory.
bool fwd_staging(const tami_diagram* d, int n_f, int* ring_chunk, size_t* smem) {
  const size_t optin = device_props(d->device).smem_optin;
  const int mode = staging_mode();
  if (mode != TAMI_STAGING_STREAMED && fwd_smem_bytes(d->hdr, n_f, 0) <= optin) {
    *ring_chunk = 0;
    *smem = fwd_smem_bytes(d->hdr, n_f, 0);
    return true;
  }
  *ring_chunk = ring_chunk_ops();
  *smem = fwd_smem_bytes(d->hdr, n_f, *ring_chunk);
  if (*smem > optin) {
    set_error("term table and tiles exceed shared memory even with the pole-DAG program streamed: " +
              std::to_string(*smem) + " bytes (at most " + std::to_string(optin) + ")");
    return false;
  }
  return true;
}

template <bool E_IN, bool SAVE, bool STREAM>
int fwd_blocks_per_sm(size_t smem) {
  cudaFuncSetAttribute(fwd_kernel<E_IN, SAVE, STREAM>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fwd_kernel<E_IN, SAVE, STREAM>, kBlock, smem) != cudaSuccess)
    per_sm = 1;
  return per_sm < 1 ? 1 : per_sm;
}

template <bool E_IN, bool SAVE>
int launch_fwd(const tami_diagram* d, FwdParams& P, cudaStream_t stream, int max_blocks) {
  size_t smem = 0;
  int chunk = 0;
  if (!fwd_staging(d, P.n_f, &chunk, &smem)) return TAMI_EUNSUPPORTED;
  P.ring_chunk = chunk;
  DeviceProps dp = device_props(d->device);
  const int per_sm = chunk ? fwd_blocks_per_sm<E_IN, SAVE, true>(smem) : fwd_blocks_per_sm<E_IN, SAVE, false>(smem);
  long long tiles = (P.n + kBlock - 1) / kBlock;
  long long grid = (long long)dp.sms * per_sm;
  if (grid > tiles) grid = tiles;
  if (max_blocks > 0 && grid > max_blocks) grid = max_blocks;
  if (grid < 1) grid = 1;
  if (chunk) fwd_kernel<E_IN, SAVE, true><<<(unsigned)grid, kBlock, smem, stream>>>(P);
  else fwd_kernel<E_IN, SAVE, false><<<(unsigned)grid, kBlock, smem, stream>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fwd_kernel launch");
  return TAMI_OK;
}

// Grid of a momentum-mode forward launch (the workspace holds one partial row per block).  When
// the generic kernel cannot stage the table (*generic_ok = false) only the specialised kernel can
// run it, whose launch is clamped to the rows of the workspace: 4 blocks per SM.
int grid_for(const tami_diagram* d, int n_f, long long n, bool* generic_ok = nullptr) {
  DeviceProps dp = device_props(d->device);
  size_t smem = 0;
  int chunk = 0;
  const bool ok = fwd_staging(d, n_f, &chunk, &smem);
  if (generic_ok) *generic_ok = ok;
  if (!ok) {
    const long long tiles = (n + kBlock - 1) / kBlock;
    return (int)std::max(1LL, std::min(tiles, 4LL * dp.sms));
  }
  // the saving instance shares the grid (one workspace size for both)
  const int per_sm = chunk ? std::min(fwd_blocks_per_sm<false, false, true>(smem), fwd_blocks_per_sm<false, true, true>(smem))
                           : std::min(fwd_blocks_per_sm<false, false, false>(smem), fwd_blocks_per_sm<false, true, false>(smem));
  long long tiles = (n + kBlock - 1) / kBlock;
  long long grid = (long long)dp.sms * per_sm;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  return (int)grid;
}

// Momentum sampling (Sec. 5.2) appends one external momentum to the sampled ones: the calls
// that sample momenta take diagrams with one external variable only.
int check_momentum(const tami_diagram* d) {
  if (d && d->n_ext != 1) {
    set_error("momentum sampling takes one external frequency and momentum (n_ext = 1)");
    return TAMI_EUNSUPPORTED;
  }
  return TAMI_OK;
}

int check_common(const tami_diagram* d, int n_f) {
  if (!d) { set_error("NULL diagram"); return TAMI_EINVAL; }
  if (!d->d_blob) { set_error("diagram not uploaded (call tami_upload)"); return TAMI_EINVAL; }
  if (n_f < 1 || n_f > kMaxFreqPerThread * kBlock) { set_error("n_f must be in [1, 2048]"); return TAMI_EINVAL; }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != d->device) { set_error("current device differs from the upload device"); return TAMI_EINVAL; }
  return TAMI_OK;
}

FwdParams make_params(const tami_diagram* d, int n_f, double beta) {
  FwdParams P;
  std::memset(&P, 0, sizeof(P));
  P.h = d->hdr;
  P.table = static_cast<const unsigned char*>(d->d_blob);
  P.n_f = n_f;
  P.beta = beta;
  P.wait_limit = wait_limit();
  return P;
}

constexpr size_t kStatusBytes = 256;

std::atomic<int> g_staging_mode{TAMI_STAGING_AUTO};
std::atomic<int> g_ring_chunk{512};
std::atomic<long long> g_wait_limit{kSpinLimit};

// Scratch of tami_forward_noalloc: a status word (first 256 bytes) followed by the per-block
// partial sums [grid][n_f][4].  It lives in the library image, so every GPU that loads the
// library holds these bytes until the process exits; no call allocates them.
constexpr size_t kNoAllocScratchBytes = 4u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch, resolved once per device with that device current
// (in host code the symbol itself is only a host-side handle, not a device address).
unsigned char* noalloc_scratch(int dev) {
  static std::mutex mu;
  static unsigned char* addr[64] = {};
  std::lock_guard<std::mutex> lk(mu);
  if (dev < 0 || dev >= 64) return nullptr;
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_error(std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return nullptr;
    }
    addr[dev] = static_cast<unsigned char*>(p);
  }
  return addr[dev];
}

}  // namespace

int staging_mode() { return g_staging_mode.load(); }
int ring_chunk_ops() { return g_ring_chunk.load(); }
long long wait_limit() { return g_wait_limit.load(); }
}  // namespace tami

using namespace tami;

extern "C" {

int tami_upload(tami_diagram* d, int device, tami_stream_t stream) {
  return guarded([&]() -> int {
  if (!d) { set_error("NULL diagram"); return TAMI_EINVAL; }
  {
    std::string why;   // never put a table the kernels could read out of range on the device
    if (!validate_table(d->hdr, d->blob.data(), d->blob.size(), &why)) {
      set_error("term table failed validation: " + why);
      return TAMI_EINVAL;
    }
  }
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
  if (d->d_blob) {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(d->device);
    cudaFree(d->d_blob);
    cudaSetDevice(device);
    d->d_blob = nullptr;
  }
  void* p = nullptr;
  e = cudaMalloc(&p, d->blob.size());
  if (e != cudaSuccess) { set_error(std::string("cudaMalloc: ") + cudaGetErrorString(e)); return TAMI_ENOMEM; }
  e = cudaMemcpyAsync(p, d->blob.data(), d->blob.size(), cudaMemcpyHostToDevice, (cudaStream_t)stream);
  if (e != cudaSuccess) { cudaFree(p); return cuda_fail(e, "cudaMemcpyAsync"); }
  e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) { cudaFree(p); return cuda_fail(e, "cudaStreamSynchronize"); }
  d->d_blob = p;
  d->device = device;
  return TAMI_OK;
  });
}

int tami_sample_energies(const tami_diagram* d, const tami_lattice* lat, uint64_t seed, uint64_t offset,
                         int64_t n, double* E, tami_stream_t stream) {
  return guarded([&]() -> int {
  int rc = check_common(d, 1);
  if (!rc) rc = check_momentum(d);
  if (rc) return rc;
  if (!lat || !E || n < 0) { set_error("bad argument"); return TAMI_EINVAL; }
  if (n == 0) return TAMI_OK;
  FwdParams P = make_params(d, 1, 1.0);
  P.t = lat->t; P.tp = lat->tp; P.mu = lat->mu; P.kx = lat->kx_ext; P.ky = lat->ky_ext;
  P.seed = seed; P.offset = offset; P.n = n;
  unsigned grid = (unsigned)((n + 255) / 256);
  sample_energies_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(P, E);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TAMI_OK : cuda_fail(e, "sample_energies launch");
  });
}

int tami_eval_energies(const tami_diagram* d, const double* E, int64_t n_e, const double* X, int n_f,
                       double beta, double* out, tami_stream_t stream) {
  return guarded([&]() -> int {
  int rc = check_common(d, n_f);
  if (rc) return rc;
  if (n_e < 0) { set_error("bad argument"); return TAMI_EINVAL; }
  if (!beta_ok(beta)) return TAMI_EINVAL;
  if (n_e == 0) return TAMI_OK;              // nothing to read or write: E and out may be NULL
  if (!E || !X || !out) { set_error("bad argument"); return TAMI_EINVAL; }
  tami_diagram* dm = const_cast<tami_diagram*>(d);
  int chunk = 0;
  size_t smem = 0;
  const bool generic_ok = fwd_staging(d, n_f, &chunk, &smem);
  const int sel = jit_select(dm, kJitKindEnergy, n_e, n_f, generic_ok);
  if (sel < 0) return -sel;
  if (sel == 1) {
    int grid = 0;
    tami_lattice none{};
    return jit_launch(dm, kJitKindEnergy, &none, 0, 0, n_e, X, n_f, beta, nullptr, out, nullptr, nullptr,
                      const_cast<double*>(E), nullptr, 1 << 30, (cudaStream_t)stream, &grid);
  }
  jit_mark_generic(dm);
  FwdParams P = make_params(d, n_f, beta);
  P.n = n_e;
  P.E_in = E;
  P.X = X;
  P.per_sample = out;
  return launch_fwd<true, false>(d, P, (cudaStream_t)stream, 0);
  });
}

int tami_forward_workspace(const tami_diagram* d, int64_t n_samples, int n_f, size_t* bytes) {
  int rc = check_common(d, n_f);
  if (rc) return rc;
  if (!bytes || n_samples < 1) { set_error("bad argument"); return TAMI_EINVAL; }
  int grid = grid_for(d, n_f, n_samples);
  *bytes = kStatusBytes + sizeof(double) * 4 * (size_t)n_f * (size_t)grid;
  return TAMI_OK;
}

int tami_forward(const tami_diagram* d, const tami_lattice* lat, uint64_t seed, uint64_t offset,
                 int64_t n_samples, const double* X, int n_f, double beta, double* mean, double* var,
                 double* per_sample, double* saved, void* workspace, size_t workspace_bytes,
                 tami_stream_t stream) {
  return guarded([&]() -> int {
  int rc = check_common(d, n_f);
  if (!rc) rc = check_momentum(d);
  if (rc) return rc;
  if (!lat || !X || !mean || !workspace || n_samples < 1) { set_error("bad argument"); return TAMI_EINVAL; }
  if (!beta_ok(beta)) return TAMI_EINVAL;
  if (((uintptr_t)workspace & 255) != 0) { set_error("workspace must be 256-byte aligned"); return TAMI_EINVAL; }
  bool generic_ok = true;
  const int grid = grid_for(d, n_f, n_samples, &generic_ok);
  const size_t need = kStatusBytes + sizeof(double) * 4 * (size_t)n_f * (size_t)grid;
  if (workspace_bytes < need) { set_error("workspace too small"); return TAMI_EINVAL; }
  tami_diagram* dm = const_cast<tami_diagram*>(d);
  const int sel = jit_select(dm, kJitKindFwd, n_samples, n_f, generic_ok);
  if (sel < 0) return -sel;
  cudaStream_t st = (cudaStream_t)stream;
  int* status = static_cast<int*>(workspace);
  double* partial = reinterpret_cast<double*>(static_cast<char*>(workspace) + kStatusBytes);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  int used_grid = grid;
  if (sel == 1) {
    rc = jit_launch(dm, kJitKindFwd, lat, seed, offset, n_samples, X, n_f, beta, nullptr, per_sample, nullptr,
                    nullptr, saved, partial, grid, st, &used_grid);
    if (rc) return rc;
  } else {
    jit_mark_generic(dm);
    FwdParams P = make_params(d, n_f, beta);
    P.t = lat->t; P.tp = lat->tp; P.mu = lat->mu; P.kx = lat->kx_ext; P.ky = lat->ky_ext;
    P.seed = seed; P.offset = offset; P.n = n_samples;
    P.X = X;
    P.per_sample = per_sample;
    P.saved = saved;
    P.partial = partial;
    P.status = status;
    rc = saved ? launch_fwd<false, true>(d, P, st, grid) : launch_fwd<false, false>(d, P, st, grid);
    if (rc) return rc;
  }
  finalize_kernel<<<n_f, kFinBlock, 0, st>>>(partial, used_grid, n_f, n_samples, status, mean, var);
  e = cudaGetLastError();
  return e == cudaSuccess ? TAMI_OK : cuda_fail(e, "finalize launch");
  });
}

// Same evaluation as tami_forward, with its scratch taken from a fixed array inside the
// library instead of a caller-supplied workspace, for callers that cannot allocate device
// memory.  See include/tami.h for the contract (size limit, first-call set-up, shared state).
int tami_forward_noalloc(const tami_diagram* d, const tami_lattice* lat, uint64_t seed, uint64_t offset,
                         int64_t n_samples, const double* X, int n_f, double beta, double* mean, double* var,
                         double* per_sample, tami_stream_t stream) {
  return guarded([&]() -> int {
  int rc = check_common(d, n_f);
  if (!rc) rc = check_momentum(d);
  if (rc) return rc;
  if (!lat || !X || !mean || n_samples < 1) { set_error("bad argument"); return TAMI_EINVAL; }
  if (!beta_ok(beta)) return TAMI_EINVAL;
  bool generic_ok = true;
  const int grid = grid_for(d, n_f, n_samples, &generic_ok);
  if (!generic_ok) return TAMI_EUNSUPPORTED;   // this call runs the generic kernel only
  const size_t need = kStatusBytes + sizeof(double) * 4 * (size_t)n_f * (size_t)grid;
  if (need > kNoAllocScratchBytes) {
    set_error("tami_forward_noalloc: needs " + std::to_string(need) + " bytes of scratch for n_f=" +
              std::to_string(n_f) + " over " + std::to_string(grid) + " blocks, above the fixed " +
              std::to_string(kNoAllocScratchBytes) + "-byte array; use tami_forward with a workspace");
    return TAMI_EINVAL;
  }
  unsigned char* base = noalloc_scratch(d->device);
  if (!base) return TAMI_ECUDA;
  cudaStream_t st = (cudaStream_t)stream;
  int* status = reinterpret_cast<int*>(base);
  double* partial = reinterpret_cast<double*>(base + kStatusBytes);
  // the status word must start at zero; the partials are fully rewritten by every launch
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  FwdParams P = make_params(d, n_f, beta);
  P.t = lat->t; P.tp = lat->tp; P.mu = lat->mu; P.kx = lat->kx_ext; P.ky = lat->ky_ext;
  P.seed = seed; P.offset = offset; P.n = n_samples;
  P.X = X;
  P.per_sample = per_sample;
  P.partial = partial;
  P.status = status;
  jit_mark_generic(const_cast<tami_diagram*>(d));
  rc = launch_fwd<false, false>(d, P, st, grid);
  if (rc) return rc;
  finalize_kernel<<<n_f, kFinBlock, 0, st>>>(partial, grid, n_f, n_samples, status, mean, var);
  e = cudaGetLastError();
  return e == cudaSuccess ? TAMI_OK : cuda_fail(e, "finalize launch");
  });
}

int tami_set_table_staging(int mode, int chunk_ops) {
  if ((mode != TAMI_STAGING_AUTO && mode != TAMI_STAGING_STREAMED) ||
      (chunk_ops != 0 && (chunk_ops < 16 || chunk_ops > 4096 || (chunk_ops & 1)))) {
    set_error("table staging: mode TAMI_STAGING_AUTO or TAMI_STAGING_STREAMED, chunk_ops 0 or even in [16, 4096]");
    return TAMI_EINVAL;
  }
  g_staging_mode.store(mode);
  if (chunk_ops) g_ring_chunk.store(chunk_ops);
  return TAMI_OK;
}

int tami_debug_set_wait_limit(int64_t first_stage_spins) {
  if (first_stage_spins < -1 || first_stage_spins > dev::kSpinLimit) {
    set_error("wait limit: -1 (default) or 0 .. 2^24");
    return TAMI_EINVAL;
  }
  g_wait_limit.store(first_stage_spins < 0 ? dev::kSpinLimit : (long long)first_stage_spins);
  return TAMI_OK;
}

int tami_selftest_exp(const double* t, int64_t n, double* y, double* em, double* y_plain, tami_stream_t stream) {
  if (!t || !y || !em || n < 0) { set_error("bad argument"); return TAMI_EINVAL; }
  if (n == 0) return TAMI_OK;
  exp_selftest_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(t, n, y, em, y_plain);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TAMI_OK : cuda_fail(e, "exp_selftest launch");
}

int tami_selftest_sincos(const double* k, int64_t n, double* s, double* c, tami_stream_t stream) {
  if (!k || !s || !c || n < 0) { set_error("bad argument"); return TAMI_EINVAL; }
  if (n == 0) return TAMI_OK;
  sincos_selftest_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(k, n, s, c);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TAMI_OK : cuda_fail(e, "sincos_selftest launch");
}

int tami_selftest_imul(const double* a, const double* b, int64_t n, double* mul, tami_stream_t stream) {
  if (!a || !b || !mul || n < 0) { set_error("bad argument"); return TAMI_EINVAL; }
  if (n == 0) return TAMI_OK;
  imul_selftest_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(a, b, n, mul);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TAMI_OK : cuda_fail(e, "imul_selftest launch");
}

int tami_selftest_imul_ftz(const double* a, const double* b, int64_t n, double* mul, tami_stream_t stream) {
  if (!a || !b || !mul || n < 0) { set_error("bad argument"); return TAMI_EINVAL; }
  if (n == 0) return TAMI_OK;
  imul_ftz_selftest_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(a, b, n, mul);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? TAMI_OK : cuda_fail(e, "imul_ftz_selftest launch");
}

int tami_selftest_fp64_rate(int variant, int blocks, int64_t trips, double* out, double* flops, tami_stream_t stream) {
  if (variant < 0 || variant >= TAMI_FP64_RATE_VARIANTS || blocks < 1 || trips < 1 || !out) {
    set_error("bad argument");
    return TAMI_EINVAL;
  }
  // m, c passed at run time so that the recurrences cannot be folded
  const cudaStream_t st = (cudaStream_t)stream;
  const long long tr = (long long)trips;
  int per_trip = 0;   // fmas per thread per trip
  switch (variant) {
    case 0: fp64_rate_kernel<8, 8, false, false><<<(unsigned)blocks, 256, 0, st>>>(tr, 0.9999999, 1e-3, out); per_trip = 64; break;
    case 1: fp64_rate_kernel<4, 8, true, false><<<(unsigned)blocks, 256, 0, st>>>(tr, 0.9999999, 1e-3, out); per_trip = 32; break;
    case 2: fp64_rate_kernel<4, 16, true, true><<<(unsigned)blocks, 256, 0, st>>>(tr, 0.9999999, 1e-3, out); per_trip = 64; break;
    default: fp64_rate_kernel<3, 16, true, false><<<(unsigned)blocks, 256, 0, st>>>(tr, 0.9999999, 1e-3, out); per_trip = 48; break;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "fp64_rate launch");
  if (flops) *flops = 2.0 * per_trip * (double)trips * 256.0 * (double)blocks;
  return TAMI_OK;
}

void tami_destroy(tami_diagram* d) {
  if (!d) return;
  jit_release(d);
  if (d->d_blob) {
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(d->device);
    cudaFree(d->d_blob);
    if (prev >= 0) cudaSetDevice(prev);
  }
  delete d;
}

}  // extern "C"
