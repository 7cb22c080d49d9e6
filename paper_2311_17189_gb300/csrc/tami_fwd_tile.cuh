// One tile of the forward evaluation (phase 1 + phase 2) and the fixed-order block reduction,
// shared by the single-diagram kernel (tami_cuda.cu) and the persistent multi-diagram kernel
// (tami_batch.cu).  Internal to the library.
#pragma once

#include "tami_device.cuh"

namespace tami {
namespace dev {

constexpr int kMaxFreqPerThread = 16;  // n_f <= kMaxFreqPerThread * kBlock

// typed views of a staged term table
struct TableView {
  const int* repl;
  const int* lm_ptr;
  const int* lm_l;
  const double* lm_c;
  const int* combo_ptr;
  const int* combo_j;
  const double* combo_c;
  const int* fseg;
  const int* fvr;
  const int* rden;
  const int* cden;
  const double* cden_a;
  const int* cden_xk;
  const double* xvec;
  const int* g1;
  const int* g1_tgt;
  const int2* ops;
  const double* leafA;
  const int* g1rd;
  const int* g2;
  const int* g2cd;
  const int* pnode;
  const int* g2node;
};

__device__ __forceinline__ TableView table_view(const unsigned char* t, const TableHeader& H) {
  TableView v;
  v.repl = reinterpret_cast<const int*>(t + H.off_repl);
  v.lm_ptr = reinterpret_cast<const int*>(t + H.off_lm_ptr);
  v.lm_l = reinterpret_cast<const int*>(t + H.off_lm_l);
  v.lm_c = reinterpret_cast<const double*>(t + H.off_lm_c);
  v.combo_ptr = reinterpret_cast<const int*>(t + H.off_combo_ptr);
  v.combo_j = reinterpret_cast<const int*>(t + H.off_combo_j);
  v.combo_c = reinterpret_cast<const double*>(t + H.off_combo_c);
  v.fseg = reinterpret_cast<const int*>(t + H.off_fseg);
  v.fvr = reinterpret_cast<const int*>(t + H.off_fv);
  v.rden = reinterpret_cast<const int*>(t + H.off_rden);
  v.cden = reinterpret_cast<const int*>(t + H.off_cden);
  v.cden_a = reinterpret_cast<const double*>(t + H.off_cden_a);
  v.cden_xk = reinterpret_cast<const int*>(t + H.off_cden_xk);
  v.xvec = reinterpret_cast<const double*>(t + H.off_xvec);
  v.g1 = reinterpret_cast<const int*>(t + H.off_g1);
  v.g1_tgt = reinterpret_cast<const int*>(t + H.off_g1_tgt);
  v.ops = reinterpret_cast<const int2*>(t + H.off_ops);
  v.leafA = reinterpret_cast<const double*>(t + H.off_leafA);
  v.g1rd = reinterpret_cast<const int*>(t + H.off_g1rd);
  v.g2 = reinterpret_cast<const int*>(t + H.off_g2);
  v.g2cd = reinterpret_cast<const int*>(t + H.off_g2cd);
  v.pnode = reinterpret_cast<const int*>(t + H.off_pnode);
  v.g2node = reinterpret_cast<const int*>(t + H.off_g2node);
  return v;
}

// The forward pole-DAG program streamed through shared memory, for tables whose program does not
// fit beside the tiles: two buffers of `chunk` ops, each filled by one cp.async.bulk completed on
// its own mbarrier; chunk c goes to buffer c & 1.  Every thread of the block walks the whole
// program in order once per tile (threads without a sample walk it too), so moving to the next
// chunk is a block-wide step: a barrier (no thread reads the old buffer any more), the refill of
// that buffer with chunk c + 2 and the wait for chunk c + 1.  Every chunk that is issued is waited
// for within the tile.  A wait that runs out sets the status word and leaves the ring failed: it
// then hands out one in-range op (slot 0, leaf 0, value 0) and issues nothing more, and the
// launch's outputs are NaN.
struct OpRing {
  const unsigned char* src;   // the program in global memory (the blob at off_ops)
  int2* buf;                  // [2][chunk] in shared memory
  unsigned long long* bar;    // [2] mbarriers, initialised by the kernel
  int* status;
  long long limit;            // bound of a wait's first stage
  int n_ops, chunk, n_chunks;
  int cur, lo, hi;            // the chunk in use and its op range
  int waits[2];               // completed waits per barrier: the next wait's parity is waits & 1
  bool failed;

  __device__ __forceinline__ void fill(int c) {   // thread 0 only
    const int o0 = c * chunk, n = min(chunk, n_ops - o0);
    // whole 16-byte units: an odd last chunk reads one op past the program (the adjoint program
    // follows it in the blob); the ring buffer holds it (chunk is even)
    bulk_issue(reinterpret_cast<unsigned char*>(buf + (c & 1) * chunk), src + 8 * (size_t)o0, (8 * n + 15) & ~15,
               nullptr, nullptr, 0, bar + (c & 1));
  }
  __device__ __forceinline__ void wait(int b) {
    const bool ok = mbar_wait(bar + b, (uint32_t)(waits[b] & 1), status, limit);
    ++waits[b];
    failed |= __syncthreads_or(!ok) != 0;
  }
  // start of a tile's walk: chunks 0 and 1 in flight, wait for chunk 0
  __device__ __forceinline__ void begin() {
    __syncthreads();
    if (!failed && threadIdx.x == 0) {
      fill(0);
      if (n_chunks > 1) fill(1);
    }
    cur = 0;
    lo = 0;
    hi = min(chunk, n_ops);
    if (!failed) wait(0);
  }
  __device__ __forceinline__ void advance() {
    __syncthreads();
    if (!failed && threadIdx.x == 0 && cur + 2 < n_chunks) fill(cur + 2);
    ++cur;
    lo = cur * chunk;
    hi = min(lo + chunk, n_ops);
    if (!failed) wait(cur & 1);
  }
  __device__ __forceinline__ int2 get(int o) {
    if (o >= hi) advance();
    if (failed) return make_int2(kOpFirst | kOpLeaf, 0);
    return buf[(cur & 1) * chunk + (o - lo)];
  }
};

// Sum over a group's terms of A_t prod FT factors, by the group's pole-tree program: one fma per
// edge of the (shared-sub-sum) tree, v[dst] = F * (leaf ? A[ref] : v[ref]) + (first ? 0 : v[dst]),
// over value slots; the root's sum is written by the group's last op.  Both operand loads use
// in-range indices, the select picks one.  STREAM: the ops come from the ring.
template <bool STREAM>
__device__ __forceinline__ double pole_tree(const TableView& T, OpRing& R, int op0, int op1, const double* fv) {
  double v[kMaxSlots];
  v[0] = 0.0;
  int dst = 0;
  for (int o = op0; o < op1; ++o) {
    const int2 op = STREAM ? R.get(o) : T.ops[o];
    dst = op.x & kOpDstMask;
    const int ref = op.x >> kOpRefShift;
    const bool leaf = op.x & kOpLeaf;
    const double a = T.leafA[leaf ? ref : 0], b = v[leaf ? 0 : ref];
    const double addend = (op.x & kOpFirst) ? 0.0 : v[dst];
    v[dst] = fma(fv[op.y], leaf ? a : b, addend);
  }
  return v[dst];
}

// Phase-2 assignment of the tile's (frequency, sample) pairs to threads.  A thread walks nf
// segments: segment i is frequency f0 + i * fstep over samples [sb, se) with stride sstep, where
// (sb, se) is (sb0, se0) for the first segment and (sb1, se1) for the others.
//   n_f divides kBlock: tpf = kBlock / n_f threads per frequency, samples strided by tpf;
//   n_f < kBlock otherwise ("balanced"): thread t takes the n_f consecutive pairs
//     [t n_f, (t+1) n_f) in frequency-major order, i.e. the end of one frequency's samples and the
//     start of the next one's (at most two segments), so every thread does n_f pairs and no warp
//     issues FP64 work for a handful of lanes;
//   n_f > kBlock: frequencies f = t, t + kBlock, ... over all samples.
struct FreqMap {
  int tpf, f0, fstep, nf, sstep, sb0, se0, sb1, se1;
  int p0;          // balanced: the first of the thread's n_f pairs
  bool balanced;
};

__device__ __forceinline__ FreqMap freq_map(int n_f, int tid) {
  FreqMap m;
  m.balanced = false;
  m.sb1 = 0;
  m.se1 = kBlock;
  if (n_f <= kBlock && kBlock % n_f == 0) {
    m.tpf = kBlock / n_f;
    m.f0 = tid / m.tpf;
    m.fstep = 1;
    m.nf = m.f0 < n_f ? 1 : 0;
    m.sb0 = tid % m.tpf;
    m.se0 = kBlock;
    m.sstep = m.tpf;
  } else if (n_f < kBlock) {
    const int p0 = tid * n_f;             // first pair, frequency-major: p = f * kBlock + s
    m.p0 = p0;
    m.balanced = true;
    m.tpf = 0;
    m.f0 = p0 / kBlock;
    m.fstep = 1;
    m.sb0 = p0 % kBlock;
    m.se0 = min(kBlock, m.sb0 + n_f);
    m.se1 = m.sb0 + n_f - kBlock;         // samples of frequency f0 + 1, if positive
    m.nf = m.se1 > 0 ? 2 : 1;
    m.sstep = 1;
  } else {
    m.tpf = 1;
    m.f0 = tid;
    m.fstep = kBlock;
    m.nf = (n_f - tid + kBlock - 1) / kBlock;
    m.sb0 = 0;
    m.se0 = kBlock;
    m.sstep = 1;
  }
  return m;
}

struct TileArgs {
  double t, tp, mu, kx, ky, beta;
  unsigned long long seed, offset;  // sample s of the tile stream is Philox counter offset + s
  long long n;                      // samples in the stream
  const double* E_in;               // energy input [n][N] or null
  double* per_sample;               // [n_f][n][2] or null
  double* saved;                    // [n_rep + 2 n_rep_ext][n] energies and dE/dK factors, or null
  int n_f;
};

// The external frequencies as the denominators see them: Y_kf = sum_q v_kq X_fq for every
// external-coefficient vector v_k of the table and frequency row f (X: [n_f][n_ext][2]), into
// Xs [n_xk][n_f][2].  A complex denominator c is then D = g_c Y_{k_c f} + b.  With one external
// (v_0 = (1)) this is a copy.  No barrier.
__device__ __forceinline__ void stage_freqs(const TableHeader& H, const TableView& T, const double* X, int n_f,
                                            double* Xs) {
  if (H.n_ext == 1) {
    for (int i = threadIdx.x; i < 2 * n_f; i += kBlock) Xs[i] = X[i];
    return;
  }
  for (int i = threadIdx.x; i < H.n_xk * n_f; i += kBlock) {
    const int k = i / n_f, f = i % n_f;
    const double* v = T.xvec + k * H.n_ext;
    const double* x = X + 2 * (size_t)f * H.n_ext;
    double re = v[0] * x[0], im = v[0] * x[1];
    for (int q = 1; q < H.n_ext; ++q) {
      re = fma(v[q], x[2 * q], re);
      im = fma(v[q], x[2 * q + 1], im);
    }
    Xs[2 * i] = re;
    Xs[2 * i + 1] = im;
  }
}

// Per-(denominator, frequency) constants of phase 2: AXI = g_c Im Y_{k_c f} and AXI2 = AXI^2, in
// shared memory [n_cden][n_f] each.  Returns whether every Re Y is zero (then Re D = b exactly).
// Ends with a barrier.
__device__ __forceinline__ bool freq_constants(const TableHeader& H, const TableView& T, const double* Xs, int n_f,
                                               double* AXI, double* AXI2) {
  int nonzero = 0;
  for (int i = threadIdx.x; i < H.n_cden * n_f; i += kBlock) {
    const int c = i / n_f, f = i % n_f;
    const double a = T.cden_a[c] * Xs[2 * (T.cden_xk[c] * n_f + f) + 1];
    AXI[i] = a;
    AXI2[i] = a * a;
  }
  for (int i = threadIdx.x; i < H.n_xk * n_f; i += kBlock) nonzero |= Xs[2 * i] != 0.0;
  return !__syncthreads_or(nonzero);
}

// Phase 2 for one (sample slot sl, frequency f): the complex reciprocals of the frequency-dependent
// denominators, the group products R_h (one complex product per node of the flattener's product
// trie) and the sum over groups of W_h R_h.  Written without data-dependent selects: on this GPU
// an FP64 instruction issued with its predicate off still occupies the FP64 pipe, so the
// imaginary-axis case is a template parameter.  A group without frequency-dependent factors sits
// first (g2_const).
template <bool XR_ZERO>
__device__ __forceinline__ void phase2_sample(const TableHeader& H, const TableView& T, const TileArgs& A, int sl,
                                              int f, const double* Xs, const double* AXI, const double* AXI2,
                                              const double* CB, const double* W, double& vr_out, double& vi_out) {
  // values: [0, n_cden) the reciprocals 1/D_c, then the product nodes
  double vre[kMaxCplxDens + kMaxProdNodes], vim[kMaxCplxDens + kMaxProdNodes];
  for (int c = 0; c < H.n_cden; ++c) {
    const double b = CB[c * kBlock + sl];
    // D = g_c Y_{k_c f} + b
    const double Dr = XR_ZERO ? b : fma(T.cden_a[c], Xs[2 * (T.cden_xk[c] * A.n_f + f)], b);
    const double r = rcp(fma(Dr, Dr, AXI2[c * A.n_f + f]));
    vre[c] = Dr * r;
    vim[c] = -AXI[c * A.n_f + f] * r;
  }
  for (int k = 0; k < H.n_pnode; ++k) {
    const int src = T.pnode[2 * k], c = T.pnode[2 * k + 1];
    const double ar = vre[src], ai = vim[src], br = vre[c], bi = vim[c];
    vre[H.n_cden + k] = fma(ar, br, -ai * bi);
    vim[H.n_cden + k] = fma(ar, bi, ai * br);
  }
  double vr = H.g2_const ? W[sl] : 0.0, vi = 0.0;
  for (int hg = H.g2_const; hg < H.n_g2; ++hg) {
    const double w = W[hg * kBlock + sl];
    const int v = T.g2node[hg];
    vr = fma(w, vre[v], vr);
    vi = fma(w, vim[v], vi);
  }
  vr_out = vr;
  vi_out = vi;
}

template <bool XR_ZERO>
__device__ __forceinline__ void phase2_loop(const TableHeader& H, const TableView& T, const TileArgs& A, long long s0,
                                            const double* Xs, const double* AXI, const double* AXI2, const double* CB,
                                            const double* W, const FreqMap& M, double (*acc)[4]);

__device__ __forceinline__ void phase2_store(const TileArgs& A, int f, long long s, double vr, double vi,
                                             double* acc) {
  if (A.per_sample) {
    double2* o = reinterpret_cast<double2*>(A.per_sample) + (size_t)f * A.n + s;
    *o = make_double2(vr, vi);
  }
  acc[0] += vr;
  acc[1] += vi;
  acc[2] = fma(vr, vr, acc[2]);
  acc[3] = fma(vi, vi, acc[3]);
}

// Shared memory per tile: Xs [n_xk][n_f][2] (from stage_freqs), AXI and AXI2 [n_cden][n_f] (from
// freq_constants), CB [n_cden][kBlock], W [n_g2][kBlock].  STREAM: the pole-DAG program comes
// through the ring R, which every thread of the block walks (a thread without a sample on zero
// energies, its values dropped by phase 2).
template <bool ENERGY_IN, bool SAVE, bool STREAM>
__device__ __forceinline__ void fwd_tile(const TableHeader& H, const TableView& T, const TileArgs& A,
                                         long long tile, const double* Xs, const double* AXI, const double* AXI2,
                                         bool xr_zero, double* CB, double* W, const FreqMap& M, double (*acc)[4],
                                         OpRing& R) {
  const int tid = threadIdx.x;
  const long long s0 = tile * kBlock;
  const double beta = A.beta;
  // ---------------------------------------------------------------- phase 1 (thread = sample)
  {
    const long long s = s0 + tid;
    const bool active = s < A.n;
    if (STREAM) R.begin();
    if (active || STREAM) {
      double E[kMaxLines];
      if (!active) {
        for (int r = 0; r < H.n_rep; ++r) E[T.repl[r]] = 0.0;
      } else if (ENERGY_IN) {
        for (int r = 0; r < H.n_rep; ++r) E[T.repl[r]] = A.E_in[s * H.N + T.repl[r]];
      } else {
        double kx[kMaxVars], ky[kMaxVars];
        const unsigned long long sg = A.offset + (unsigned long long)s;
        for (int l = 0; l < H.m; ++l) {
          uint32_t c[4] = {(uint32_t)sg, (uint32_t)(sg >> 32), (uint32_t)l, 0u};
          philox4x32_10(c, (uint32_t)A.seed, (uint32_t)(A.seed >> 32));
          kx[l] = to_momentum(c[0], c[1]);
          ky[l] = to_momentum(c[2], c[3]);
        }
        kx[H.m] = A.kx;
        ky[H.m] = A.ky;
        auto line_momentum = [&](int r, double& ax, double& ay) {
          ax = 0.0;
          ay = 0.0;
          for (int q = T.lm_ptr[r]; q < T.lm_ptr[r + 1]; ++q) {
            const double cf = T.lm_c[q];
            const int l = T.lm_l[q];
            ax = fma(cf, kx[l], ax);
            ay = fma(cf, ky[l], ay);
          }
        };
        int r = 0;
        if (SAVE) {   // for the adjoint: the lines carrying k_ext also give their dE/dK factors
          for (; r < H.n_rep_ext; ++r) {
            double ax, ay, gx, gy;
            line_momentum(r, ax, ay);
            E[T.repl[r]] = line_energy_grad(ax, ay, A.t, A.tp, A.mu, gx, gy);
            A.saved[(size_t)(H.n_rep + 2 * r) * A.n + s] = gx;
            A.saved[(size_t)(H.n_rep + 2 * r + 1) * A.n + s] = gy;
          }
        }
        for (; r < H.n_rep; ++r) {
          double ax, ay;
          line_momentum(r, ax, ay);
          E[T.repl[r]] = line_energy(ax, ay, A.t, A.tp, A.mu);
        }
        if (SAVE)
          for (int q = 0; q < H.n_rep; ++q) A.saved[(size_t)q * A.n + s] = E[T.repl[q]];
      }
      double x[kMaxCombos];
      for (int u = 0; u < H.n_combo; ++u) {
        double v = 0.0;
        for (int q = T.combo_ptr[u]; q < T.combo_ptr[u + 1]; ++q) v = fma(T.combo_c[q], E[T.combo_j[q]], v);
        x[u] = v;
      }
      double fv[kMaxFermiValues];
      for (int b = 0; b < H.n_fseg_bose; ++b) fermi_segment<true, false>(T.fseg + 8 * b, T.fvr, x, beta, fv, nullptr);
      for (int b = H.n_fseg_bose; b < H.n_fseg; ++b)
        fermi_segment<false, false>(T.fseg + 8 * b, T.fvr, x, beta, fv, nullptr);
      double rr[kMaxRealDens];
      for (int i = 0; i < H.n_rden; ++i) rr[i] = rcp(x[T.rden[2 * i]]);
      int cur = T.g1_tgt[0];
      double wacc = 0.0;
      for (int gi = 0; gi < H.n_g1; ++gi) {
        const int tg = T.g1_tgt[gi];
        if (tg != cur) { W[cur * kBlock + tid] = wacc; wacc = 0.0; cur = tg; }
        double ft = pole_tree<STREAM>(T, R, T.g1[4 * gi], T.g1[4 * gi + 1], fv);
        for (int q = T.g1[4 * gi + 2]; q < T.g1[4 * gi + 3]; ++q) {
          const double r = rr[T.g1rd[2 * q]];
          for (int pw = T.g1rd[2 * q + 1]; pw > 0; --pw) ft *= r;
        }
        wacc += ft;
      }
      W[cur * kBlock + tid] = wacc;
      for (int c = 0; c < H.n_cden; ++c) {
        const double xv = x[T.cden[2 * c]];
        CB[c * kBlock + tid] = T.cden[2 * c + 1] > 0 ? xv : -xv;
      }
    }
  }
  __syncthreads();
  // ---------------------------------------------------------------- phase 2 ((f, s) pairs)
  if (xr_zero) phase2_loop<true>(H, T, A, s0, Xs, AXI, AXI2, CB, W, M, acc);
  else phase2_loop<false>(H, T, A, s0, Xs, AXI, AXI2, CB, W, M, acc);
  __syncthreads();
}

// Two samples per iteration give the FP64 pipe two independent dependency chains; the sums are
// still taken sample by sample, in the same order.
// Swap the running sums of the thread's two frequencies (selects, no FP64 work).
__device__ __forceinline__ void swap_sums(bool sw, double* a, double* b) {
  for (int k = 0; k < 4; ++k) {
    const double x = a[k], y = b[k];
    a[k] = sw ? y : x;
    b[k] = sw ? x : y;
  }
}

template <bool XR_ZERO>
__device__ __forceinline__ void phase2_loop(const TableHeader& H, const TableView& T, const TileArgs& A, long long s0,
                                            const double* Xs, const double* AXI, const double* AXI2, const double* CB,
                                            const double* W, const FreqMap& M, double (*acc)[4]) {
  if (M.balanced) {
    // One flat loop over the thread's n_f pairs p = p0 .. p0 + n_f - 1 (frequency p / kBlock, slot
    // p % kBlock), the same trip count in every lane.  The sums go to cur, which holds the
    // current frequency's sums: when p reaches the next frequency (slot 0) cur and oth swap.
    // Slots past the end of the sample stream (last tile) are evaluated on whatever the tile
    // buffers hold and dropped.
    double cur[4], oth[4];
    for (int k = 0; k < 4; ++k) { cur[k] = acc[0][k]; oth[k] = acc[1][k]; }
    bool crossed = false;
    int j = 0;
    for (; j + 1 < A.n_f; j += 2) {
      const int pa = M.p0 + j, pb = pa + 1;
      const int fa = pa / kBlock, sla = pa % kBlock, fb = pb / kBlock, slb = pb % kBlock;
      double ar, ai, br, bi;
      phase2_sample<XR_ZERO>(H, T, A, sla, fa, Xs, AXI, AXI2, CB, W, ar, ai);
      phase2_sample<XR_ZERO>(H, T, A, slb, fb, Xs, AXI, AXI2, CB, W, br, bi);
      const bool sa = sla == 0 && j > 0, sb = slb == 0;
      swap_sums(sa, cur, oth);
      crossed |= sa;
      if (s0 + sla < A.n) phase2_store(A, fa, s0 + sla, ar, ai, cur);
      swap_sums(sb, cur, oth);
      crossed |= sb;
      if (s0 + slb < A.n) phase2_store(A, fb, s0 + slb, br, bi, cur);
    }
    if (j < A.n_f) {
      const int pa = M.p0 + j, fa = pa / kBlock, sla = pa % kBlock;
      double ar, ai;
      phase2_sample<XR_ZERO>(H, T, A, sla, fa, Xs, AXI, AXI2, CB, W, ar, ai);
      const bool sa = sla == 0 && j > 0;
      swap_sums(sa, cur, oth);
      crossed |= sa;
      if (s0 + sla < A.n) phase2_store(A, fa, s0 + sla, ar, ai, cur);
    }
    swap_sums(crossed, cur, oth);     // back to acc[0] = frequency f0, acc[1] = f0 + 1
    for (int k = 0; k < 4; ++k) { acc[0][k] = cur[k]; acc[1][k] = oth[k]; }
    return;
  }
  for (int fi = 0; fi < M.nf; ++fi) {
    const int f = M.f0 + fi * M.fstep;
    int sl = fi ? M.sb1 : M.sb0;
    const int se = fi ? M.se1 : M.se0;
    for (; sl + M.sstep < se && s0 + sl + M.sstep < A.n; sl += 2 * M.sstep) {
      double ar, ai, br, bi;
      phase2_sample<XR_ZERO>(H, T, A, sl, f, Xs, AXI, AXI2, CB, W, ar, ai);
      phase2_sample<XR_ZERO>(H, T, A, sl + M.sstep, f, Xs, AXI, AXI2, CB, W, br, bi);
      phase2_store(A, f, s0 + sl, ar, ai, acc[fi]);
      phase2_store(A, f, s0 + sl + M.sstep, br, bi, acc[fi]);
    }
    for (; sl < se && s0 + sl < A.n; sl += M.sstep) {
      double ar, ai;
      phase2_sample<XR_ZERO>(H, T, A, sl, f, Xs, AXI, AXI2, CB, W, ar, ai);
      phase2_store(A, f, s0 + sl, ar, ai, acc[fi]);
    }
  }
}

// Sum the per-thread accumulators of the block in a fixed order into out[n_f][4].
// red: 4 * kBlock doubles of shared memory.  Ends with a barrier.
__device__ __forceinline__ void block_reduce_store(const FreqMap& M, int n_f, double (*acc)[4], double* red,
                                                   double* out) {
  const int tid = threadIdx.x;
  if (M.balanced) {
    // Frequency f is covered by threads tlo..thi (their pair ranges meet [f kBlock, (f+1) kBlock)).
    // Its sum, in this order: the second segment of tlo when tlo starts on frequency f - 1, then
    // the first segments of the threads that start on f, in thread order.
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    const int tlo = tid < n_f ? (tid * kBlock) / n_f : 0;
    const int thi = tid < n_f ? (tid * kBlock + kBlock - 1) / n_f : -1;
    for (int k = 0; k < 4; ++k) red[k * kBlock + tid] = M.nf > 1 ? acc[1][k] : 0.0;
    __syncthreads();
    if (tid < n_f && (tlo * n_f) / kBlock != tid)
      for (int k = 0; k < 4; ++k) s[k] = red[k * kBlock + tlo];
    __syncthreads();
    for (int k = 0; k < 4; ++k) red[k * kBlock + tid] = acc[0][k];
    __syncthreads();
    if (tid < n_f) {
      for (int t = tlo; t <= thi; ++t)
        if ((t * n_f) / kBlock == tid)
          for (int k = 0; k < 4; ++k) s[k] += red[k * kBlock + t];
      for (int k = 0; k < 4; ++k) out[tid * 4 + k] = s[k];
    }
  } else if (n_f <= kBlock) {
    for (int k = 0; k < 4; ++k) red[k * kBlock + tid] = acc[0][k];
    __syncthreads();
    if (tid < n_f) {
      for (int k = 0; k < 4; ++k) {
        double s = 0.0;
        for (int j = 0; j < M.tpf; ++j) s += red[k * kBlock + tid * M.tpf + j];
        out[tid * 4 + k] = s;
      }
    }
  } else {
    for (int fi = 0; fi < M.nf; ++fi) {
      const int f = M.f0 + fi * M.fstep;
      for (int k = 0; k < 4; ++k) out[f * 4 + k] = acc[fi][k];
    }
  }
  __syncthreads();
}

}  // namespace dev
}  // namespace tami
