// Adjoint of the Monte Carlo evaluation (sm_103a, FP64).  For an upstream gradient g_f of the
// sample means Sigma_f (one complex number per external frequency) it returns
//   dSigma_f/dX_f                          (the derivative along the external frequency; with
//                                           X = omega + i Gamma this is dSigma/domega, whose real
//                                           part gives the quasiparticle weight),
//   d/domega_f  Re conj(g_f) Sigma_f,
//   d/dtheta    Re sum_f conj(g_f) Sigma_f  for theta = mu, kx_ext, ky_ext.
// The paper defines the forward evaluation (Sec. 2.3, Sec. 5.2); it has no adjoint.
//
// One thread per sample, every phase sample-major: the forward quantities of phase 1 are
// recomputed (combinations, Fermi values and their next derivative, the pole DAG keeping every
// node's value, group weights) from line energies that are either recomputed from the momenta or
// read from rows the forward saved; phase 2 runs over all frequencies and collects dv/dX, the
// adjoints of the group weights and of the frequency-dependent denominator energies; a reverse
// sweep pushes those back through the pole DAG, the Fermi/Bose derivatives (d/dx P_k = P_{k+1}),
// the energy combinations and the dispersion (dE/dmu = 1, dE/dk_ext = -alpha_ext * G).  Term
// products are recomputed, never stored.  The fused instance (tami_forward_backward) also forms
// each sample's value and the forward's sums in phase 2.  Reductions are in a fixed order.
#include <algorithm>
#include <cstring>

#include "tami_device.cuh"
#include "tami_internal.h"

namespace tami {
namespace {

using namespace dev;

// per-thread capacities of the adjoint (checked before launch)
constexpr int kBwCombos = 64, kBwFv = 128, kBwRden = 32, kBwCden = 32, kBwG1 = 128, kBwG2 = 64;
constexpr int kBwFreq = 256, kBwNodes = 1024, kBwG2cd = 256;

struct BwdParams {
  TableHeader h;
  const unsigned char* table;
  double t, tp, mu, kx, ky;
  unsigned long long seed, offset;
  long long n;
  const double* X;       // [n_f][2]
  const double* G;       // [n_f][2] upstream gradient
  int n_f;
  double beta;
  double* ps_dX;         // [n_f][n][2] or null
  double* ps_grad;       // [n][3] or null
  const double* saved;   // [n_rep + 2 n_rep_ext][n] from tami_forward, or null (recompute)
  double* ps_v;          // fused pass: [n_f][n][2] each sample's value, or null
  double* partial;       // [grid][2 n_f + 3]
  int* status;
  long long wait_limit;   // bound of the first stage of the staging wait
};

// Values each block reduces: dv/dX [n_f][2], the three parameter gradients and, in the fused pass,
// the forward's sums [n_f][4] (Re, Im, Re^2, Im^2).
__host__ __device__ __forceinline__ int bwd_nval(int n_f, bool fwd) { return 2 * n_f + 3 + (fwd ? 4 * n_f : 0); }

// Shared memory: table | X, G [n_f][2] | AXI, AXI2 [n_cden][n_f] | red [4 warps][nval].  The table
// part is [0, off_ops) followed by the adjoint program [off_opsb, bytes) (the forward program is
// not staged).
__host__ __device__ __forceinline__ size_t bwd_table_smem(const TableHeader& h) {
  return (size_t)h.off_ops + (size_t)(h.bytes - h.off_opsb);
}

__host__ __device__ __forceinline__ size_t bwd_smem_bytes(const TableHeader& h, int n_f, bool fwd) {
  return bwd_table_smem(h) +
         sizeof(double) * ((4 + 2 * (size_t)h.n_cden) * n_f + 4 * (size_t)bwd_nval(n_f, fwd));
}

// Phase 2 of the adjoint for one sample over all frequencies: the reciprocals, the group products
// R_h (the flattener's product trie), the weight adjoints Wb_h += Re(conj g R_h), U_d = sum_h p W_h R_h
// (pW = p W_h per group factor, formed once per sample), Z_d = r_d U_d, dv/dX = -sum_d a_d Z_d and
// the denominator-energy adjoints bb_d -= Re(conj g Z_d).  As in the forward, no data-dependent
// selects around FP64 work (predicated-off FP64 instructions still cost FP64-pipe time): the R = 1
// group is group 0 (its weight adjoint, sum_f Re g_f, is the same for every sample: the caller
// sets it from a per-block sum) and the imaginary-axis case is a template parameter.
template <bool XR_ZERO, bool FWD>
__device__ __forceinline__ void bwd_phase2(const TableHeader& H, int n_f, long long s, const BwdParams& P,
                                           const double* Xs, const double* Gs, const double* AXI, const double* AXI2,
                                           const double* cden_a, const int* g2, const int* g2cd, const int* pnode,
                                           const int* g2node, const double* pW, const double* b, const double* W2,
                                           double* Wb2, double* bb, double* accX, double* accV) {
  for (int f = 0; f < n_f; ++f) {
    const double Xr = Xs[2 * f], gr = Gs[2 * f], gim = Gs[2 * f + 1], ngr = -gr, ngi = -gim;
    double vre[kBwCden + kMaxProdNodes], vim[kBwCden + kMaxProdNodes], U_re[kBwCden], U_im[kBwCden];
    for (int c = 0; c < H.n_cden; ++c) {
      const double Dr = XR_ZERO ? b[c] : fma(cden_a[c], Xr, b[c]);
      const double r = rcp(fma(Dr, Dr, AXI2[c * n_f + f]));
      vre[c] = Dr * r;
      vim[c] = -AXI[c * n_f + f] * r;
      U_re[c] = 0.0;
      U_im[c] = 0.0;
    }
    for (int k = 0; k < H.n_pnode; ++k) {
      const int src = pnode[2 * k], c = pnode[2 * k + 1];
      const double ar = vre[src], ai = vim[src], br = vre[c], bi = vim[c];
      vre[H.n_cden + k] = fma(ar, br, -ai * bi);
      vim[H.n_cden + k] = fma(ar, bi, ai * br);
    }
    double vr = 0.0, vi = 0.0;                    // fused pass: the sample's value sum_h W_h R_h
    if (FWD) vr = H.g2_const ? W2[0] : 0.0;
    for (int h = H.g2_const; h < H.n_g2; ++h) {
      const int v = g2node[h];
      const double Rr = vre[v], Ri = vim[v];
      if (FWD) {
        vr = fma(W2[h], Rr, vr);
        vi = fma(W2[h], Ri, vi);
      }
      Wb2[h] = fma(gr, Rr, fma(gim, Ri, Wb2[h]));
      for (int q = g2[h]; q < g2[h + 1]; ++q) {
        const int cc = g2cd[2 * q];
        U_re[cc] = fma(pW[q], Rr, U_re[cc]);
        U_im[cc] = fma(pW[q], Ri, U_im[cc]);
      }
    }
    double dvr = 0.0, dvi = 0.0;
    for (int c = 0; c < H.n_cden; ++c) {
      const double Zr = fma(vre[c], U_re[c], -vim[c] * U_im[c]);
      const double Zi = fma(vre[c], U_im[c], vim[c] * U_re[c]);
      dvr = fma(-cden_a[c], Zr, dvr);
      dvi = fma(-cden_a[c], Zi, dvi);
      bb[c] = fma(ngr, Zr, fma(ngi, Zi, bb[c]));
    }
    accX[2 * f] += dvr;
    accX[2 * f + 1] += dvi;
    if (P.ps_dX) {
      double2* o = reinterpret_cast<double2*>(P.ps_dX) + (size_t)f * P.n + s;
      *o = make_double2(dvr, dvi);
    }
    if (FWD) {
      accV[4 * f] += vr;
      accV[4 * f + 1] += vi;
      accV[4 * f + 2] = fma(vr, vr, accV[4 * f + 2]);
      accV[4 * f + 3] = fma(vi, vi, accV[4 * f + 3]);
      if (P.ps_v) reinterpret_cast<double2*>(P.ps_v)[(size_t)f * P.n + s] = make_double2(vr, vi);
    }
  }
}

// Resident blocks per SM that the register allocation must allow (the kernel's arrays live in
// local memory; 8 blocks fit in 64 registers without spills).
#ifndef TAMI_BWD_MIN_BLOCKS
#define TAMI_BWD_MIN_BLOCKS 8
#endif

// SAVED: read the forward's saved rows instead of recomputing the energies.  FWD: the fused pass,
// which also forms each sample's value and the forward's sums (mean, variance) in phase 2.
template <bool SAVED, bool FWD>
__global__ void __launch_bounds__(kBlock, TAMI_BWD_MIN_BLOCKS) bwd_kernel(const BwdParams P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const TableHeader& H = P.h;
  const int tid = threadIdx.x;
  if (!stage_table(smem, P.table, H.off_ops, P.status, P.wait_limit, P.table + H.off_opsb, H.bytes - H.off_opsb))
    return;
  const int n_f = P.n_f;
  double* Xs = reinterpret_cast<double*>(smem + bwd_table_smem(H));
  double* Gs = Xs + 2 * n_f;
  double* AXI = Gs + 2 * n_f;
  double* AXI2 = AXI + H.n_cden * n_f;
  double* red = AXI2 + H.n_cden * n_f;       // [4 warps][nval]
  for (int i = tid; i < 2 * n_f; i += kBlock) { Xs[i] = P.X[i]; Gs[i] = P.G[i]; }

  const int* repl = reinterpret_cast<const int*>(smem + H.off_repl);
  const int* lm_ptr = reinterpret_cast<const int*>(smem + H.off_lm_ptr);
  const int* lm_l = reinterpret_cast<const int*>(smem + H.off_lm_l);
  const double* lm_c = reinterpret_cast<const double*>(smem + H.off_lm_c);
  const double* rep_aext = reinterpret_cast<const double*>(smem + H.off_rep_aext);
  const int* combo_ptr = reinterpret_cast<const int*>(smem + H.off_combo_ptr);
  const int* combo_j = reinterpret_cast<const int*>(smem + H.off_combo_j);
  const double* combo_c = reinterpret_cast<const double*>(smem + H.off_combo_c);
  const int* fseg = reinterpret_cast<const int*>(smem + H.off_fseg);
  const int* fvr = reinterpret_cast<const int*>(smem + H.off_fv);
  const int* rden = reinterpret_cast<const int*>(smem + H.off_rden);
  const int* cden = reinterpret_cast<const int*>(smem + H.off_cden);
  const double* cden_a = reinterpret_cast<const double*>(smem + H.off_cden_a);
  const int* g1 = reinterpret_cast<const int*>(smem + H.off_g1);
  const int* g1_tgt = reinterpret_cast<const int*>(smem + H.off_g1_tgt);
  const int2* opsb = reinterpret_cast<const int2*>(smem + H.off_ops);   // staged right after [0, off_ops)
  const int* g1_node = reinterpret_cast<const int*>(smem + H.off_g1_node);
  const double* leafA = reinterpret_cast<const double*>(smem + H.off_leafA);
  const int* g1rd = reinterpret_cast<const int*>(smem + H.off_g1rd);
  const int* g2 = reinterpret_cast<const int*>(smem + H.off_g2);
  const int* g2cd = reinterpret_cast<const int*>(smem + H.off_g2cd);
  const double* g2cd_p = reinterpret_cast<const double*>(smem + H.off_g2cd_p);
  const int* pnode = reinterpret_cast<const int*>(smem + H.off_pnode);
  const int* g2node = reinterpret_cast<const int*>(smem + H.off_g2node);

  double accX[2 * kBwFreq], accV[FWD ? 4 * kBwFreq : 1];
  for (int i = 0; i < 2 * n_f; ++i) accX[i] = 0.0;
  if (FWD)
    for (int i = 0; i < 4 * n_f; ++i) accV[i] = 0.0;
  double gmu = 0.0, gkx = 0.0, gky = 0.0;
  __shared__ double s_gsum;                  // sum_f Re g_f in frequency order: the R = 1 group's Wb
  __syncthreads();
  bool xr_zero;
  {
    int nonzero = 0;
    for (int i = tid; i < H.n_cden * n_f; i += kBlock) {
      const double a = cden_a[i / n_f] * Xs[2 * (i % n_f) + 1];
      AXI[i] = a;
      AXI2[i] = a * a;
    }
    for (int f = tid; f < n_f; f += kBlock) nonzero |= Xs[2 * f] != 0.0;
    if (tid == 0) {
      double g = 0.0;
      for (int f = 0; f < n_f; ++f) g += Gs[2 * f];
      s_gsum = g;
    }
    xr_zero = !__syncthreads_or(nonzero);
  }

  const double beta = P.beta;
  const long long n_tiles = (P.n + kBlock - 1) / kBlock;
  for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
    const long long s = tile * kBlock + tid;
    if (s >= P.n) continue;
    // ------------------------------------------------------------ forward recomputation
    // line energies, and for the lines carrying k_ext the factors G of dE/dK = -G: read from the
    // forward's saved rows, or recomputed from the momenta exactly as the forward forms them
    double E[kMaxLines], Gx[kMaxLines], Gy[kMaxLines];
    if (SAVED) {
      for (int r = 0; r < H.n_rep; ++r) E[repl[r]] = P.saved[(size_t)r * P.n + s];
      for (int r = 0; r < H.n_rep_ext; ++r) {
        Gx[r] = P.saved[(size_t)(H.n_rep + 2 * r) * P.n + s];
        Gy[r] = P.saved[(size_t)(H.n_rep + 2 * r + 1) * P.n + s];
      }
    } else {
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
      auto line_momentum = [&](int r, double& ax, double& ay) {
        ax = 0.0;
        ay = 0.0;
        for (int q = lm_ptr[r]; q < lm_ptr[r + 1]; ++q) {
          const double cf = lm_c[q];
          const int l = lm_l[q];
          ax = fma(cf, kx[l], ax);
          ay = fma(cf, ky[l], ay);
        }
      };
      for (int r = 0; r < H.n_rep_ext; ++r) {
        double ax, ay;
        line_momentum(r, ax, ay);
        E[repl[r]] = line_energy_grad(ax, ay, P.t, P.tp, P.mu, Gx[r], Gy[r]);
      }
      for (int r = H.n_rep_ext; r < H.n_rep; ++r) {
        double ax, ay;
        line_momentum(r, ax, ay);
        E[repl[r]] = line_energy(ax, ay, P.t, P.tp, P.mu);
      }
    }
    double x[kBwCombos];
    for (int u = 0; u < H.n_combo; ++u) {
      double v = 0.0;
      for (int q = combo_ptr[u]; q < combo_ptr[u + 1]; ++q) v = fma(combo_c[q], E[combo_j[q]], v);
      x[u] = v;
    }
    double fv[kBwFv], fvd[kBwFv];
    for (int b = 0; b < H.n_fseg_bose; ++b) fermi_segment<true, true>(fseg + 8 * b, fvr, x, beta, fv, fvd);
    for (int b = H.n_fseg_bose; b < H.n_fseg; ++b) fermi_segment<false, true>(fseg + 8 * b, fvr, x, beta, fv, fvd);
    double rr[kBwRden];
    for (int i = 0; i < H.n_rden; ++i) rr[i] = rcp(x[rden[2 * i]]);
    // pole trees (adjoint encoding: one slot per node), keeping every node's value for the reverse
    double W1[kBwG1], W2[kBwG2], val[kBwNodes];
    for (int h = 0; h < H.n_g2; ++h) W2[h] = 0.0;
    val[0] = 0.0;
    for (int gi = 0; gi < H.n_g1; ++gi) {
      for (int o = g1[4 * gi]; o < g1[4 * gi + 1]; ++o) {
        const int2 op = opsb[o];
        const int dst = op.x & kOpbDstMask, ref = op.y >> kOpbRefShift;
        const bool leaf = op.x & kOpbLeaf;
        const double a = leafA[leaf ? ref : 0], b = val[leaf ? 0 : ref];
        const double addend = (op.x & kOpbFirst) ? 0.0 : val[dst];
        val[dst] = fma(fv[op.y & kOpbFvMask], leaf ? a : b, addend);
      }
      double ft = val[g1_node[gi]];
      for (int q = g1[4 * gi + 2]; q < g1[4 * gi + 3]; ++q) {
        const double r = rr[g1rd[2 * q]];
        for (int pw = g1rd[2 * q + 1]; pw > 0; --pw) ft *= r;
      }
      W1[gi] = ft;
      W2[g1_tgt[gi]] += ft;
    }
    double b[kBwCden];
    for (int c = 0; c < H.n_cden; ++c) {
      const double xv = x[cden[2 * c]];
      b[c] = cden[2 * c + 1] > 0 ? xv : -xv;
    }
    // ------------------------------------------------------------ phase 2 over frequencies
    double Wb2[kBwG2], bb[kBwCden], pW[kBwG2cd];
    for (int h = 0; h < H.n_g2; ++h) {
      Wb2[h] = 0.0;
      for (int q = g2[h]; q < g2[h + 1]; ++q) pW[q] = g2cd_p[q] * W2[h];
    }
    for (int c = 0; c < H.n_cden; ++c) bb[c] = 0.0;
    if (xr_zero)
      bwd_phase2<true, FWD>(H, n_f, s, P, Xs, Gs, AXI, AXI2, cden_a, g2, g2cd, pnode, g2node, pW, b, W2, Wb2, bb,
                            accX, accV);
    else
      bwd_phase2<false, FWD>(H, n_f, s, P, Xs, Gs, AXI, AXI2, cden_a, g2, g2cd, pnode, g2node, pW, b, W2, Wb2, bb,
                             accX, accV);
    if (H.g2_const) Wb2[0] = s_gsum;             // R = 1: sum_f Re(conj g_f * 1), as the loop would add it
    // ------------------------------------------------------------ reverse sweep
    double xbar[kBwCombos], fvbar[kBwFv];
    for (int u = 0; u < H.n_combo; ++u) xbar[u] = 0.0;
    for (int v = 0; v < H.n_fv; ++v) fvbar[v] = 0.0;
    for (int c = 0; c < H.n_cden; ++c) {
      const int u = cden[2 * c];
      xbar[u] += cden[2 * c + 1] > 0 ? bb[c] : -bb[c];
    }
    for (int gi = H.n_g1 - 1; gi >= 0; --gi) {
      const double wb = Wb2[g1_tgt[gi]];
      double RR = 1.0;
      for (int q = g1[4 * gi + 2]; q < g1[4 * gi + 3]; ++q) {
        const int i = g1rd[2 * q];
        const int pw = g1rd[2 * q + 1];
        for (int k = 0; k < pw; ++k) RR *= rr[i];
        // W1 = FT prod rr^p and rr = 1/x:  dW1/dx = -p rr W1
        xbar[rden[2 * i]] -= wb * W1[gi] * (double)pw * rr[i];
      }
      // pole tree, reverse: for the edge v[dst] += F * operand,
      //   Fbar += operand * vbar[dst]  and, for inner edges,  vbar[ref] += F * vbar[dst];
      // a node's run of leaf edges shares vbar[dst].  Post order puts every use of a node after its
      // own edges, so walking backwards completes vbar of a node before its edges are reached.
      const int o0 = g1[4 * gi], nb = g1_node[gi], ne = g1_node[gi + 1];
      double bar[kBwNodes];
      for (int k = nb + 1; k < ne; ++k) bar[k] = 0.0;
      bar[nb] = wb * RR;
      for (int o = g1[4 * gi + 1] - 1; o >= o0;) {
        const int2 op = opsb[o];
        const double pb = bar[op.x & kOpbDstMask];
        if (op.x & kOpbLeaf) {
          const int run = max((op.x >> kOpbRunShift) & 255, 1);   // >= 1: the walk always advances
          for (int i = 0; i < run; ++i) {
            const int2 q = opsb[o - i];
            const int qf = q.y & kOpbFvMask;
            fvbar[qf] = fma(leafA[q.y >> kOpbRefShift], pb, fvbar[qf]);
          }
          o -= run;
        } else {
          const int ref = op.y >> kOpbRefShift, f = op.y & kOpbFvMask;
          fvbar[f] = fma(val[ref], pb, fvbar[f]);
          bar[ref] = fma(fv[f], pb, bar[ref]);
          --o;
        }
      }
    }
    for (int bse = 0; bse < H.n_fseg; ++bse) {
      const int* sgm = fseg + 8 * bse;
      double acc = 0.0;
      for (int v = sgm[2]; v < sgm[4]; ++v) {
        const double d = fvbar[v] * fvd[v];
        acc += fvr[2 * v] > 0 ? d : -d;
      }
      xbar[sgm[0]] += acc;
    }
    double Ebar[kMaxLines];
    for (int r = 0; r < H.n_rep; ++r) Ebar[repl[r]] = 0.0;
    for (int u = 0; u < H.n_combo; ++u)
      for (int q = combo_ptr[u]; q < combo_ptr[u + 1]; ++q) Ebar[combo_j[q]] = fma(xbar[u], combo_c[q], Ebar[combo_j[q]]);
    double mub = 0.0, kxb = 0.0, kyb = 0.0;
    for (int r = 0; r < H.n_rep; ++r) mub += Ebar[repl[r]];
    for (int r = 0; r < H.n_rep_ext; ++r) {
      const double eb = Ebar[repl[r]];
      const double ae = rep_aext[r];
      // dE/dK = -G = -(2t + 4t' cos K_perp) sin K,  dK/dk_ext = alpha_ext
      kxb = fma(-eb * ae, Gx[r], kxb);
      kyb = fma(-eb * ae, Gy[r], kyb);
    }
    gmu += mub;
    gkx += kxb;
    gky += kyb;
    if (P.ps_grad) {
      P.ps_grad[3 * s] = mub;
      P.ps_grad[3 * s + 1] = kxb;
      P.ps_grad[3 * s + 2] = kyb;
    }
  }
  // -------------------------------------------------------------- block reduction
  const int nval = bwd_nval(n_f, FWD);
  const int warp = tid >> 5, lane = tid & 31;
  for (int i = 0; i < nval; ++i) {
    double v = i < 2 * n_f ? accX[i] : (i == 2 * n_f ? gmu : (i == 2 * n_f + 1 ? gkx : gky));
    if (FWD && i >= 2 * n_f + 3) v = accV[i - 2 * n_f - 3];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp * nval + i] = v;
  }
  __syncthreads();
  for (int i = tid; i < nval; i += kBlock) {
    double v = 0.0;
    for (int w = 0; w < kBlock / 32; ++w) v += red[w * nval + i];
    P.partial[(size_t)blockIdx.x * nval + i] = v;
  }
}

__global__ void __launch_bounds__(kFinBlock) bwd_finalize_kernel(const double* partial, int n_blocks, int n_f, long long n, const double* G,
                                    const int* status, double* dX, double* grad_omega, double* grad_params) {
  // block i < n_f: dSigma/dX_i (two columns); block n_f: the three parameter gradients
  __shared__ double sh[3][kFinBlock];
  const int i = blockIdx.x;
  const int nval = 2 * n_f + 3;
  const int c0 = i < n_f ? 2 * i : 2 * n_f;
  double s[3] = {0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < n_blocks; b += kFinBlock) {
    const double* p = partial + (size_t)b * nval + c0;
    s[0] += p[0];
    s[1] += p[1];
    if (i == n_f) s[2] += p[2];
  }
  fixed_tree_sum<3>(s, sh);
  if (threadIdx.x != 0) return;
  const bool bad = status && *status != 0;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  if (i < n_f) {
    double re = s[0] / (double)n, im = s[1] / (double)n;
    if (bad) re = im = nan;
    if (dX) { dX[2 * i] = re; dX[2 * i + 1] = im; }
    if (grad_omega) grad_omega[i] = bad ? nan : fma(G[2 * i], re, G[2 * i + 1] * im);
  } else if (grad_params) {
    for (int k = 0; k < 3; ++k) grad_params[k] = bad ? nan : s[k] / (double)n;
  }
}

// Whether the generic adjoint kernel can take the table: its per-thread arrays and shared memory.
bool bwd_generic_ok(const tami_diagram* d, int n_f, bool fwd) {
  const TableHeader& h = d->hdr;
  if (h.n_combo > kBwCombos || h.n_fv > kBwFv || h.n_rden > kBwRden || h.n_cden > kBwCden ||
      h.n_g1 > kBwG1 || h.n_g2 > kBwG2 || h.n_nodes > kBwNodes || h.n_g2cd > kBwG2cd) {
    set_error("term table exceeds the generic adjoint kernel's per-sample capacities: " + std::to_string(h.n_combo) +
              " combinations (" + std::to_string(kBwCombos) + "), " + std::to_string(h.n_fv) + " Fermi values (" +
              std::to_string(kBwFv) + "), " + std::to_string(h.n_rden) + " real denominators (" +
              std::to_string(kBwRden) + "), " + std::to_string(h.n_cden) + " complex denominators (" +
              std::to_string(kBwCden) + "), " + std::to_string(h.n_g1) + " groups (" + std::to_string(kBwG1) +
              "), " + std::to_string(h.n_g2) + " frequency groups (" + std::to_string(kBwG2) + "), " +
              std::to_string(h.n_nodes) + " DAG nodes (" + std::to_string(kBwNodes) + "), " +
              std::to_string(h.n_g2cd) + " phase-2 factors (" + std::to_string(kBwG2cd) + ")");
    return false;
  }
  if (bwd_smem_bytes(h, n_f, fwd) > device_props(d->device).smem_optin) {
    set_error("term table and frequencies exceed shared memory in the generic adjoint kernel");
    return false;
  }
  return true;
}

// Grid of an adjoint launch (the workspace holds its partial rows).  A table the generic kernel
// cannot take (*generic_ok = false) runs only on the specialised kernel, whose launch is clamped to
// the workspace's rows: 4 blocks per SM.
int bwd_grid(const tami_diagram* d, int n_f, long long n, size_t* smem_out, bool fwd, bool* generic_ok = nullptr) {
  DeviceProps dp = device_props(d->device);
  const size_t smem = bwd_smem_bytes(d->hdr, n_f, fwd);
  if (smem_out) *smem_out = smem;
  const bool ok = bwd_generic_ok(d, n_f, fwd);
  if (generic_ok) *generic_ok = ok;
  if (!ok) {
    const long long tiles = (n + kBlock - 1) / kBlock;
    return (int)std::max(1LL, std::min(tiles, 4LL * dp.sms));
  }
  int per_sm = 0;
  if (fwd) {
    cudaFuncSetAttribute(bwd_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bwd_kernel<false, true>, kBlock, smem) != cudaSuccess)
      per_sm = 1;
  } else {
    // one grid for both adjoint instances (saved rows or recomputation), so that their reductions
    // group the samples alike and the results agree bit for bit
    cudaFuncSetAttribute(bwd_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaFuncSetAttribute(bwd_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int per_sm_saved = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bwd_kernel<false, false>, kBlock, smem) != cudaSuccess)
      per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_saved, bwd_kernel<true, false>, kBlock, smem) !=
        cudaSuccess)
      per_sm_saved = 1;
    if (per_sm_saved < per_sm) per_sm = per_sm_saved;
  }
  if (per_sm < 1) per_sm = 1;
  long long tiles = (n + kBlock - 1) / kBlock;
  long long grid = (long long)dp.sms * per_sm;
  if (grid > tiles) grid = tiles;
  if (grid < 1) grid = 1;
  return (int)grid;
}

// The fused pass's final reduction: block f < n_f sums dv/dX_f and the forward's four sums of f,
// block n_f the three parameter gradients; fixed tree order.
__global__ void __launch_bounds__(kFinBlock) fused_finalize_kernel(const double* partial, int n_blocks, int n_f,
                                                                  long long n, const double* G, const int* status,
                                                                  double* mean, double* var, double* dX,
                                                                  double* grad_omega, double* grad_params) {
  __shared__ double sh[6][kFinBlock];
  const int i = blockIdx.x;
  const int nval = bwd_nval(n_f, true);
  double s[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < n_blocks; b += kFinBlock) {
    const double* p = partial + (size_t)b * nval;
    if (i < n_f) {
      s[0] += p[2 * i];
      s[1] += p[2 * i + 1];
      for (int k = 0; k < 4; ++k) s[2 + k] += p[2 * n_f + 3 + 4 * i + k];
    } else {
      for (int k = 0; k < 3; ++k) s[k] += p[2 * n_f + k];
    }
  }
  fixed_tree_sum<6>(s, sh);
  if (threadIdx.x != 0) return;
  const bool bad = status && *status != 0;
  const double nan = __longlong_as_double(0x7ff8000000000000ll), nn = (double)n;
  if (i < n_f) {
    const double re = bad ? nan : s[0] / nn, im = bad ? nan : s[1] / nn;
    if (dX) { dX[2 * i] = re; dX[2 * i + 1] = im; }
    if (grad_omega) grad_omega[i] = bad ? nan : fma(G[2 * i], re, G[2 * i + 1] * im);
    const double mr = s[2] / nn, mi = s[3] / nn;
    const double vr = n > 1 ? (s[4] - s[2] * mr) / (nn - 1.0) : 0.0;
    const double vi = n > 1 ? (s[5] - s[3] * mi) / (nn - 1.0) : 0.0;
    mean[2 * i] = bad ? nan : mr;
    mean[2 * i + 1] = bad ? nan : mi;
    if (var) { var[2 * i] = bad ? nan : vr; var[2 * i + 1] = bad ? nan : vi; }
  } else if (grad_params) {
    for (int k = 0; k < 3; ++k) grad_params[k] = bad ? nan : s[k] / nn;
  }
}

int bwd_check(const tami_diagram* d, int n_f) {
  if (!d) { set_error("NULL diagram"); return TAMI_EINVAL; }
  if (!d->d_blob) { set_error("diagram not uploaded (call tami_upload)"); return TAMI_EINVAL; }
  if (n_f < 1 || n_f > kBwFreq) { set_error("n_f must be in [1, 256] for the adjoint"); return TAMI_EINVAL; }
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != d->device) { set_error("current device differs from the upload device"); return TAMI_EINVAL; }
  const TableHeader& h = d->hdr;
  if (h.n_ext != 1) { set_error("momentum sampling takes one external frequency and momentum (n_ext = 1)"); return TAMI_EUNSUPPORTED; }
  if (h.max_der > 4) { set_error("the adjoint needs derivative orders up to 4"); return TAMI_EUNSUPPORTED; }
  return TAMI_OK;
}

constexpr size_t kBwStatusBytes = 256;

}  // namespace
}  // namespace tami

using namespace tami;

extern "C" {

int tami_backward_workspace(const tami_diagram* d, int64_t n_samples, int n_f, size_t* bytes) {
  int rc = bwd_check(d, n_f);
  if (rc) return rc;
  if (!bytes || n_samples < 1) { set_error("bad argument"); return TAMI_EINVAL; }
  const int grid = bwd_grid(d, n_f, n_samples, nullptr, false);
  *bytes = kBwStatusBytes + sizeof(double) * (size_t)bwd_nval(n_f, false) * (size_t)grid;
  return TAMI_OK;
}

int tami_forward_backward_workspace(const tami_diagram* d, int64_t n_samples, int n_f, size_t* bytes) {
  int rc = bwd_check(d, n_f);
  if (rc) return rc;
  if (!bytes || n_samples < 1) { set_error("bad argument"); return TAMI_EINVAL; }
  const int grid = bwd_grid(d, n_f, n_samples, nullptr, true);
  *bytes = kBwStatusBytes + sizeof(double) * (size_t)bwd_nval(n_f, true) * (size_t)grid;
  return TAMI_OK;
}

int tami_backward(const tami_diagram* d, const tami_lattice* lat, uint64_t seed, uint64_t offset,
                  int64_t n_samples, const double* X, int n_f, double beta, const double* gout,
                  double* dsigma_dX, double* grad_X_re, double* grad_params, double* per_sample_dX,
                  double* per_sample_grads, const double* saved, void* workspace, size_t workspace_bytes,
                  tami_stream_t stream) {
  return guarded([&]() -> int {
  int rc = bwd_check(d, n_f);
  if (rc) return rc;
  if (!lat || !X || !gout || !workspace || n_samples < 1) { set_error("bad argument"); return TAMI_EINVAL; }
  if (!beta_ok(beta)) return TAMI_EINVAL;
  if (((uintptr_t)workspace & 255) != 0) { set_error("workspace must be 256-byte aligned"); return TAMI_EINVAL; }
  size_t smem = 0;
  bool generic_ok = true;
  const int grid = bwd_grid(d, n_f, n_samples, &smem, false, &generic_ok);
  const std::string generic_why = generic_ok ? std::string() : std::string(tami_last_error());
  const size_t need = kBwStatusBytes + sizeof(double) * (size_t)bwd_nval(n_f, false) * (size_t)grid;
  if (workspace_bytes < need) { set_error("workspace too small"); return TAMI_EINVAL; }
  tami_diagram* dm = const_cast<tami_diagram*>(d);
  const int sel = jit_select(dm, kJitKindBwd, n_samples, n_f, generic_ok);
  if (sel < 0) return -sel;
  if (sel == 0 && !generic_ok) { set_error(generic_why); return TAMI_EUNSUPPORTED; }
  cudaStream_t st = (cudaStream_t)stream;
  int* status = static_cast<int*>(workspace);
  double* partial = reinterpret_cast<double*>(static_cast<char*>(workspace) + kBwStatusBytes);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  int used_grid = grid;
  if (sel == 1) {
    rc = jit_launch(dm, kJitKindBwd, lat, seed, offset, n_samples, X, n_f, beta, gout, nullptr, per_sample_dX,
                    per_sample_grads, const_cast<double*>(saved), partial, grid, st, &used_grid);
    if (rc) return rc;
  } else {
    jit_mark_generic(dm);
    BwdParams P;
    std::memset(&P, 0, sizeof(P));
    P.h = d->hdr;
    P.table = static_cast<const unsigned char*>(d->d_blob);
    P.t = lat->t; P.tp = lat->tp; P.mu = lat->mu; P.kx = lat->kx_ext; P.ky = lat->ky_ext;
    P.seed = seed; P.offset = offset; P.n = n_samples;
    P.X = X; P.G = gout; P.n_f = n_f; P.beta = beta;
    P.ps_dX = per_sample_dX; P.ps_grad = per_sample_grads;
    P.saved = saved;
    P.partial = partial; P.status = status;
    P.wait_limit = wait_limit();
    if (saved) bwd_kernel<true, false><<<grid, kBlock, smem, st>>>(P);
    else bwd_kernel<false, false><<<grid, kBlock, smem, st>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "bwd_kernel launch");
  }
  bwd_finalize_kernel<<<n_f + 1, kFinBlock, 0, st>>>(partial, used_grid, n_f, n_samples, gout, status,
                                                              dsigma_dX, grad_X_re, grad_params);
  e = cudaGetLastError();
  return e == cudaSuccess ? TAMI_OK : cuda_fail(e, "bwd finalize launch");
  });
}

int tami_forward_backward(const tami_diagram* d, const tami_lattice* lat, uint64_t seed, uint64_t offset,
                          int64_t n_samples, const double* X, int n_f, double beta, const double* gout, double* mean,
                          double* var, double* per_sample, double* dsigma_dX, double* grad_X_re, double* grad_params,
                          double* per_sample_dX, double* per_sample_grads, void* workspace, size_t workspace_bytes,
                          tami_stream_t stream) {
  return guarded([&]() -> int {
  int rc = bwd_check(d, n_f);
  if (rc) return rc;
  if (!lat || !X || !gout || !mean || !workspace || n_samples < 1) { set_error("bad argument"); return TAMI_EINVAL; }
  if (!beta_ok(beta)) return TAMI_EINVAL;
  if (((uintptr_t)workspace & 255) != 0) { set_error("workspace must be 256-byte aligned"); return TAMI_EINVAL; }
  size_t smem = 0;
  bool generic_ok = true;
  const int grid = bwd_grid(d, n_f, n_samples, &smem, true, &generic_ok);
  const std::string generic_why = generic_ok ? std::string() : std::string(tami_last_error());
  const size_t need = kBwStatusBytes + sizeof(double) * (size_t)bwd_nval(n_f, true) * (size_t)grid;
  if (workspace_bytes < need) { set_error("workspace too small"); return TAMI_EINVAL; }
  // the diagram's specialised kernel (compiled once and cached with it) or the generic one
  tami_diagram* dm = const_cast<tami_diagram*>(d);
  const int sel = jit_select(dm, kJitKindFused, n_samples, n_f, generic_ok);
  if (sel < 0) return -sel;
  if (sel == 0 && !generic_ok) { set_error(generic_why); return TAMI_EUNSUPPORTED; }
  cudaStream_t st = (cudaStream_t)stream;
  int* status = static_cast<int*>(workspace);
  double* partial = reinterpret_cast<double*>(static_cast<char*>(workspace) + kBwStatusBytes);
  cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
  int used_grid = grid;
  if (sel == 1) {
    rc = jit_launch(dm, kJitKindFused, lat, seed, offset, n_samples, X, n_f, beta, gout, per_sample, per_sample_dX,
                    per_sample_grads, nullptr, partial, grid, st, &used_grid);
    if (rc) return rc;
  } else {
    jit_mark_generic(dm);
    BwdParams P;
    std::memset(&P, 0, sizeof(P));
    P.h = d->hdr;
    P.table = static_cast<const unsigned char*>(d->d_blob);
    P.t = lat->t; P.tp = lat->tp; P.mu = lat->mu; P.kx = lat->kx_ext; P.ky = lat->ky_ext;
    P.seed = seed; P.offset = offset; P.n = n_samples;
    P.X = X; P.G = gout; P.n_f = n_f; P.beta = beta;
    P.ps_dX = per_sample_dX; P.ps_grad = per_sample_grads; P.ps_v = per_sample;
    P.partial = partial; P.status = status;
    P.wait_limit = wait_limit();
    bwd_kernel<false, true><<<grid, kBlock, smem, st>>>(P);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "fused kernel launch");
  }
  fused_finalize_kernel<<<n_f + 1, kFinBlock, 0, st>>>(partial, used_grid, n_f, n_samples, gout, status, mean, var,
                                                       dsigma_dX, grad_X_re, grad_params);
  e = cudaGetLastError();
  return e == cudaSuccess ? TAMI_OK : cuda_fail(e, "fused finalize launch");
  });
}

}  // extern "C"
