// Schwarz alternating procedure (Sec. 3, Figs. 2-3) as one kernel per colour.
//
// The lattice is cut into blocks of bs[0] x ... x bs[3] sites; block colour =
// parity of the sum of its block coordinates (an even number of blocks per
// direction, so blocks of one colour never touch).  One CTA handles one block
// of the requested colour, one thread per block site:
//
//   1. r_i = (rho - D phi)_i with the full stencil (neighbours in the
//      other-colour blocks carry the latest boundary values; phi of this
//      colour is only written by this CTA, at the end);
//   2. MR steps on the block operator D_i (Dirichlet: hops leaving the block
//      dropped, clover kept), with r_i in shared memory ([component][site]
//      for conflict-free neighbour reads), p = D_i r in registers:
//      omega = <p, r> / <p, p>, x += omega r, r -= omega p;
//      the adaptive variant (Sec. 3.2) leaves the loop when, after at least
//      4 steps, ||r|| > alpha ||r_prev||, when ||r|| grew, or when ||r|| fell
//      below tol = res ||eta|| / n_blocks; every decision is block-uniform;
//   3. phi_i += x.
// sap_smem_eo_kernel replaces 2 by MR steps on the block's even-odd Schur
// complement (see below).  Block reductions are binary64.  Arithmetic and storage binary32.
// sap_smem_kernel (the default) stages the block's links and clover in
// shared memory first; sap_kernel reads them from global memory.
#include "oq_internal.h"
#include "oq_kernels.h"
#include "hop_impl.cuh"

namespace oq {

struct SapArgs {
  Geom g;
  int bs[4];
  int nb[4];
  int colour;
  const void* links;   // binary32 packed links
  const void* clov;    // binary32 packed clover
  const void* clov_inv;  // binary32 packed inverse clover (even-odd block solver)
  const char* rho;     // packed binary32 full field
  char* phi;           // packed binary32 full field, updated in place
  long half_bytes;
  int nmr;
  int adaptive;
  float alpha;
  double tol;          // adaptive exit 3 (absolute block norm)
  unsigned* mr_steps;  // accumulated MR steps over all blocks (may be null)
};

__device__ __forceinline__ void load_smem(const float* sm, int nsite, int t, Spinor<float>& s) {
#pragma unroll
  for (int k = 0; k < 12; ++k) s.c[k / 3][k % 3] = cx<float>{sm[(2 * k) * nsite + t], sm[(2 * k + 1) * nsite + t]};
}
__device__ __forceinline__ void store_smem(float* sm, int nsite, int t, const Spinor<float>& s) {
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    sm[(2 * k) * nsite + t] = s.c[k / 3][k % 3].re;
    sm[(2 * k + 1) * nsite + t] = s.c[k / 3][k % 3].im;
  }
}

// The block sums of an MR step, result in every thread.  The three sums
// that give the MR coefficient omega = <D p, r> / <D p, D p> are binary32
// (a preconditioner coefficient: a tree of warp shuffles, then the warp
// partials in a fixed order; ~5e-7 relative for 256 sites); binary64
// arithmetic runs at 1/64 of the binary32 rate on GB300, and these sums with
// a binary64 division per thread had kept its FP64 pipe 36 % busy.  The
// adaptive exit tests keep one binary64 sum (block_sum1).
__device__ __forceinline__ void block_sum3(float& a, float& b, float& c, double* red_d) {
  float* red = reinterpret_cast<float*>(red_d);
  a = warp_sum_f(a);
  b = warp_sum_f(b);
  c = warp_sum_f(c);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    red[3 * w] = a;
    red[3 * w + 1] = b;
    red[3 * w + 2] = c;
  }
  __syncthreads();
  a = b = c = 0.f;
  for (int k = 0; k < nw; ++k) {
    a += red[3 * k];
    b += red[3 * k + 1];
    c += red[3 * k + 2];
  }
}
__device__ __forceinline__ double block_sum1(double a, double* red) {
  a = warp_sum(a);
  const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = a;
  __syncthreads();
  a = 0.0;
  for (int k = 0; k < nw; ++k) a += red[k];
  return a;
}

// in-block hop along +mu / -mu from smem (Dirichlet: outside neighbours dropped)
template <int FMT, int MU>
__device__ __forceinline__ void block_hop(const SapArgs& a, const float* sm, int nsite, int t, const int l[4],
                                          const int x[4], int p, long i, Spinor<float>& acc) {
  int stride = 1;
  for (int nu = 3; nu > MU; --nu) stride *= a.bs[nu];
  if (l[MU] + 1 < a.bs[MU]) {
    Spinor<float> nb;
    load_smem(sm, nsite, t + stride, nb);
    HalfSpinor<float> h, r;
    project<MU, -1>(nb, h);
    Su3<float> u;
    load_link<float, FMT>(a.links, a.g.Vh, p, MU, i, u);
    su3_mul(u, h, r);
    accum_reconstruct<MU, -1>(acc, r, -0.5f);
  }
  if (l[MU] > 0) {
    Spinor<float> nb;
    load_smem(sm, nsite, t - stride, nb);
    HalfSpinor<float> h, r;
    project<MU, +1>(nb, h);
    int y[4] = {x[0], x[1], x[2], x[3]};
    y[MU] -= 1;
    Su3<float> u;
    load_link<float, FMT>(a.links, a.g.Vh, 1 - p, MU, eo_index(a.g, y), u);
    su3_dag_mul(u, h, r);
    accum_reconstruct<MU, +1>(acc, r, -0.5f);
  }
}

// MINB = 2 caps registers so that two 256-thread CTAs fit on an SM (a few
// spills to L1), MINB = 1 lets the compiler use ~200 registers (one CTA)
template <int FMT, int MINB>
__global__ void __launch_bounds__(256, MINB) sap_kernel(const SapArgs a) {
  extern __shared__ float sm[];
  const int nsite = a.bs[0] * a.bs[1] * a.bs[2] * a.bs[3];
  double* red = reinterpret_cast<double*>(sm + 24 * nsite);
  const int t = threadIdx.x;
  const bool act = t < nsite;
  // which block: the blockIdx.x-th block of colour a.colour
  const int half3 = a.nb[3] / 2;
  int row = blockIdx.x / half3;
  const int m = blockIdx.x % half3;
  const int bc2 = row % a.nb[2];
  row /= a.nb[2];
  const int bc1 = row % a.nb[1];
  const int bc0 = row / a.nb[1];
  const int bc3 = 2 * m + ((a.colour + bc0 + bc1 + bc2) & 1);
  int l[4], x[4];
  {
    int tt = act ? t : 0;
    l[3] = tt % a.bs[3];
    tt /= a.bs[3];
    l[2] = tt % a.bs[2];
    tt /= a.bs[2];
    l[1] = tt % a.bs[1];
    l[0] = tt / a.bs[1];
  }
  x[0] = bc0 * a.bs[0] + l[0];
  x[1] = bc1 * a.bs[1] + l[1];
  x[2] = bc2 * a.bs[2] + l[2];
  x[3] = bc3 * a.bs[3] + l[3];
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  const long i = eo_index(a.g, x);

  // 1. block residual r = rho - D phi (full stencil)
  Spinor<float> r;
  if (act) {
    HopArgs ha;
    ha.g = a.g;
    ha.links = a.links;
    const char* nbf = a.phi + (long)(1 - p) * a.half_bytes;
    Spinor<float> acc;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc.c[s][c] = cx<float>{0.f, 0.f};
    hop_dir<P_F32, FMT, 0, false>(ha, nbf, p, i, x, acc, -0.5f);
    hop_dir<P_F32, FMT, 1, false>(ha, nbf, p, i, x, acc, -0.5f);
    hop_dir<P_F32, FMT, 2, false>(ha, nbf, p, i, x, acc, -0.5f);
    hop_dir<P_F32, FMT, 3, false>(ha, nbf, p, i, x, acc, -0.5f);
    Spinor<float> ph, aph, rh;
    load_spinor<P_F32>(a.phi + (long)p * a.half_bytes, a.g.Vh, i, ph);
    clover_apply<float>(a.clov, a.g.Vh, p, i, ph, aph);
    load_spinor<P_F32>(a.rho + (long)p * a.half_bytes, a.g.Vh, i, rh);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) r.c[s][c] = rh.c[s][c] - (aph.c[s][c] + acc.c[s][c]);
    store_smem(sm, nsite, t, r);
  }
  double n0 = 0.0;
  if (a.adaptive) {
    if (act) n0 = site_norm2(r);
    n0 = block_sum1(n0, red);  // also the barrier after the block residual is stored
  } else {
    __syncthreads();
  }
  double rn_prev = sqrt(n0);

  // 2. MR on D_i
  Spinor<float> xs;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) xs.c[s][c] = cx<float>{0.f, 0.f};
  int steps = 0;
  for (int k = 1; k <= a.nmr; ++k) {
    Spinor<float> pv;
    float pr_re = 0.f, pr_im = 0.f, pp = 0.f;
    if (act) {
      Spinor<float> own;
      load_smem(sm, nsite, t, own);
      clover_apply<float>(a.clov, a.g.Vh, p, i, own, pv);
      block_hop<FMT, 0>(a, sm, nsite, t, l, x, p, i, pv);
      block_hop<FMT, 1>(a, sm, nsite, t, l, x, p, i, pv);
      block_hop<FMT, 2>(a, sm, nsite, t, l, x, p, i, pv);
      block_hop<FMT, 3>(a, sm, nsite, t, l, x, p, i, pv);
      float ar = 0.f, ai = 0.f, a2 = 0.f;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cx<float> q = pv.c[s][c], v = own.c[s][c];
          ar += q.re * v.re + q.im * v.im;
          ai += q.re * v.im - q.im * v.re;
          a2 += q.re * q.re + q.im * q.im;
        }
      pr_re = ar;
      pr_im = ai;
      pp = a2;
    }
    block_sum3(pr_re, pr_im, pp, red);  // contains __syncthreads: all neighbour reads done
    float om_re = 0.f, om_im = 0.f;
    if (pp > 0.f) {
      om_re = pr_re / pp;
      om_im = pr_im / pp;
    }
    const cx<float> om{om_re, om_im};
    double n1 = 0.0;
    if (act) {
      Spinor<float> own;
      load_smem(sm, nsite, t, own);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cfma(xs.c[s][c], om, own.c[s][c]);
          own.c[s][c] = own.c[s][c] - om * pv.c[s][c];
        }
      store_smem(sm, nsite, t, own);
      n1 = site_norm2(own);
    }
    steps = k;
    if (a.adaptive) {
      n1 = block_sum1(n1, red);
      const double rn_new = sqrt(n1);
      if ((k >= 4 && rn_new > (double)a.alpha * rn_prev) || rn_new > rn_prev || rn_new < a.tol) break;
      rn_prev = rn_new;
    } else {
      __syncthreads();  // the updated residual is read by the neighbours next step
    }
  }
  // 3. phi_i += x
  if (act) {
    char* pp = a.phi + (long)p * a.half_bytes;
    Spinor<float> ph;
    load_spinor<P_F32>(pp, a.g.Vh, i, ph);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) ph.c[s][c] = ph.c[s][c] + xs.c[s][c];
    store_spinor<P_F32>(pp, a.g.Vh, i, ph);
  }
  if (a.mr_steps && t == 0) atomicAdd(a.mr_steps, (unsigned)steps);
}

// ---------------------------------------------------------------------------
// The same block solve with the block's operands staged in shared memory
// once: the 4 forward links of every block site (18 reals, rebuilt from 12
// where stored compressed) and its two clover blocks.  The MR steps then
// read only shared memory (the residual, the links, the clover) instead of
// fetching ~670 bytes per site and step from L2.  Static MR (not adaptive)
// needs no norm reduction per step, only the barrier before the residual is
// read again.  Shared memory: 24 + 4*18 + 72 floats per block site.
// ---------------------------------------------------------------------------
struct SapSm {
  float* r;        // [24][nsite] block residual
  float2* u;       // [mu][9][nsite] forward links, 18 reals
  float4* a;       // [18][nsite] clover (two blocks: 6 diagonal + 15 complex each)
  int nsite;
};

__device__ __forceinline__ void sm_link(const SapSm& m, int mu, int t, Su3<float>& u) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const float2 v = m.u[(mu * 9 + k) * m.nsite + t];
    u.m[k / 3][k % 3] = cx<float>{v.x, v.y};
  }
}

__device__ __forceinline__ void sm_clover(const SapSm& m, int t, const Spinor<float>& in, Spinor<float>& out) {
  const cx<float>* v = &in.c[0][0];
  cx<float>* o = &out.c[0][0];
#pragma unroll
  for (int b = 0; b < 2; ++b) {
    float r[36];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const float4 w = m.a[(9 * b + k) * m.nsite + t];
      r[4 * k] = w.x;
      r[4 * k + 1] = w.y;
      r[4 * k + 2] = w.z;
      r[4 * k + 3] = w.w;
    }
    const cx<float>* x = v + 6 * b;
    cx<float>* y = o + 6 * b;
#pragma unroll
    for (int r0 = 0; r0 < 6; ++r0) y[r0] = r[r0] * x[r0];
    int k = 0;
#pragma unroll
    for (int r0 = 0; r0 < 6; ++r0)
#pragma unroll
      for (int c0 = r0 + 1; c0 < 6; ++c0) {
        const cx<float> off{r[6 + 2 * k], r[7 + 2 * k]};
        cfma(y[r0], off, x[c0]);
        cfmac(y[c0], off, x[r0]);
        ++k;
      }
  }
}

// in-block hop along +mu / -mu, all operands from shared memory
template <int MU>
__device__ __forceinline__ void sm_block_hop(const SapSm& m, const int bs[4], int t, const int l[4],
                                             Spinor<float>& acc) {
  int stride = 1;
  for (int nu = 3; nu > MU; --nu) stride *= bs[nu];
  if (l[MU] + 1 < bs[MU]) {
    Spinor<float> nb;
    load_smem(m.r, m.nsite, t + stride, nb);
    HalfSpinor<float> h, r;
    project<MU, -1>(nb, h);
    Su3<float> u;
    sm_link(m, MU, t, u);
    su3_mul(u, h, r);
    accum_reconstruct<MU, -1>(acc, r, -0.5f);
  }
  if (l[MU] > 0) {
    Spinor<float> nb;
    load_smem(m.r, m.nsite, t - stride, nb);
    HalfSpinor<float> h, r;
    project<MU, +1>(nb, h);
    Su3<float> u;
    sm_link(m, MU, t - stride, u);  // U_mu(x - mu): the forward link of the site below
    su3_dag_mul(u, h, r);
    accum_reconstruct<MU, +1>(acc, r, -0.5f);
  }
}

template <int FMT>
__global__ void __launch_bounds__(256) sap_smem_kernel(const SapArgs a) {
  extern __shared__ float4 sm4[];
  const int nsite = a.bs[0] * a.bs[1] * a.bs[2] * a.bs[3];
  SapSm m;
  m.nsite = nsite;
  m.a = sm4;                                                   // 18 float4 per site
  m.u = reinterpret_cast<float2*>(sm4 + 18 * nsite);           // 36 float2 per site
  m.r = reinterpret_cast<float*>(m.u + 36 * nsite);            // 24 floats per site
  double* red = reinterpret_cast<double*>(m.r + 24 * nsite);
  const int t = threadIdx.x;
  const bool act = t < nsite;
  const int half3 = a.nb[3] / 2;
  int row = blockIdx.x / half3;
  const int mb = blockIdx.x % half3;
  const int bc2 = row % a.nb[2];
  row /= a.nb[2];
  const int bc1 = row % a.nb[1];
  const int bc0 = row / a.nb[1];
  const int bc3 = 2 * mb + ((a.colour + bc0 + bc1 + bc2) & 1);
  int l[4], x[4];
  {
    int tt = act ? t : 0;
    l[3] = tt % a.bs[3];
    tt /= a.bs[3];
    l[2] = tt % a.bs[2];
    tt /= a.bs[2];
    l[1] = tt % a.bs[1];
    l[0] = tt / a.bs[1];
  }
  x[0] = bc0 * a.bs[0] + l[0];
  x[1] = bc1 * a.bs[1] + l[1];
  x[2] = bc2 * a.bs[2] + l[2];
  x[3] = bc3 * a.bs[3] + l[3];
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;
  const long i = eo_index(a.g, x);

  Spinor<float> r;
  if (act) {
    // stage the operands: forward links (18 reals) and clover of this site
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      Su3<float> u;
      load_link<float, FMT>(a.links, a.g.Vh, p, mu, i, u);
#pragma unroll
      for (int k = 0; k < 9; ++k) m.u[(mu * 9 + k) * nsite + t] = make_float2(u.m[k / 3][k % 3].re, u.m[k / 3][k % 3].im);
    }
    const float4* q = reinterpret_cast<const float4*>(a.clov) + (long)p * 18 * a.g.Vh;
#pragma unroll
    for (int k = 0; k < 18; ++k) m.a[k * nsite + t] = __ldg(q + k * a.g.Vh + i);
    // 1. block residual r = rho - D phi (full stencil, global operands)
    HopArgs ha;
    ha.g = a.g;
    ha.links = a.links;
    const char* nbf = a.phi + (long)(1 - p) * a.half_bytes;
    Spinor<float> acc;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc.c[s][c] = cx<float>{0.f, 0.f};
    hop_dir<P_F32, FMT, 0, false>(ha, nbf, p, i, x, acc, -0.5f);
    hop_dir<P_F32, FMT, 1, false>(ha, nbf, p, i, x, acc, -0.5f);
    hop_dir<P_F32, FMT, 2, false>(ha, nbf, p, i, x, acc, -0.5f);
    hop_dir<P_F32, FMT, 3, false>(ha, nbf, p, i, x, acc, -0.5f);
    Spinor<float> ph, aph, rh;
    load_spinor<P_F32>(a.phi + (long)p * a.half_bytes, a.g.Vh, i, ph);
    clover_apply<float>(a.clov, a.g.Vh, p, i, ph, aph);
    load_spinor<P_F32>(a.rho + (long)p * a.half_bytes, a.g.Vh, i, rh);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) r.c[s][c] = rh.c[s][c] - (aph.c[s][c] + acc.c[s][c]);
    store_smem(m.r, nsite, t, r);
  }
  double n0 = 0.0;
  if (a.adaptive) {
    if (act) n0 = site_norm2(r);
    n0 = block_sum1(n0, red);  // also the barrier after the staging
  } else {
    __syncthreads();
  }
  double rn_prev = sqrt(n0);

  // 2. MR on D_i, operands in shared memory
  Spinor<float> xs;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) xs.c[s][c] = cx<float>{0.f, 0.f};
  int steps = 0;
  for (int k = 1; k <= a.nmr; ++k) {
    Spinor<float> pv;
    float pr_re = 0.f, pr_im = 0.f, pp = 0.f;
    if (act) {
      Spinor<float> own;
      load_smem(m.r, nsite, t, own);
      sm_clover(m, t, own, pv);
      sm_block_hop<0>(m, a.bs, t, l, pv);
      sm_block_hop<1>(m, a.bs, t, l, pv);
      sm_block_hop<2>(m, a.bs, t, l, pv);
      sm_block_hop<3>(m, a.bs, t, l, pv);
      float ar = 0.f, ai = 0.f, a2 = 0.f;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cx<float> q2 = pv.c[s][c], v = own.c[s][c];
          ar += q2.re * v.re + q2.im * v.im;
          ai += q2.re * v.im - q2.im * v.re;
          a2 += q2.re * q2.re + q2.im * q2.im;
        }
      pr_re = ar;
      pr_im = ai;
      pp = a2;
    }
    block_sum3(pr_re, pr_im, pp, red);  // contains __syncthreads: all neighbour reads done
    float om_re = 0.f, om_im = 0.f;
    if (pp > 0.f) {
      om_re = pr_re / pp;
      om_im = pr_im / pp;
    }
    const cx<float> om{om_re, om_im};
    double n1 = 0.0;
    if (act) {
      Spinor<float> own;
      load_smem(m.r, nsite, t, own);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cfma(xs.c[s][c], om, own.c[s][c]);
          own.c[s][c] = own.c[s][c] - om * pv.c[s][c];
        }
      store_smem(m.r, nsite, t, own);
      n1 = site_norm2(own);
    }
    steps = k;
    if (a.adaptive) {
      n1 = block_sum1(n1, red);
      const double rn_new = sqrt(n1);
      if ((k >= 4 && rn_new > (double)a.alpha * rn_prev) || rn_new > rn_prev || rn_new < a.tol) break;
      rn_prev = rn_new;
    } else {
      __syncthreads();  // the updated residual is read by the neighbours next step
    }
  }
  // 3. phi_i += x
  if (act) {
    char* pp = a.phi + (long)p * a.half_bytes;
    Spinor<float> ph;
    load_spinor<P_F32>(pp, a.g.Vh, i, ph);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) ph.c[s][c] = ph.c[s][c] + xs.c[s][c];
    store_spinor<P_F32>(pp, a.g.Vh, i, ph);
  }
  if (a.mr_steps && t == 0) atomicAdd(a.mr_steps, (unsigned)steps);
}

// ---------------------------------------------------------------------------
// Even-odd reduced block solver (openQCD's choice for SAP, Sec. 3): per block
//   rhat_e = r_e - D_eo A_oo^{-1} r_o,
//   MR steps on Dhat_i = A_ee - D_eo A_oo^{-1} D_oe (even block sites),
//   delta_o = A_oo^{-1} (r_o - D_oe delta_e),
// D_eo, D_oe the in-block hops.  The shared field holds the even vector at
// even sites and the odd intermediate at odd sites, so one MR step is two
// half passes (odd threads, then even threads) separated by a barrier; the
// staged clover is A at even and A^{-1} at odd sites.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void zero_spinor(Spinor<float>& v) {
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) v.c[s][c] = cx<float>{0.f, 0.f};
}

// The block's sites are held parity-sorted: position k < nsite/2 is the
// block-local-even site with in-block lexicographic index n = 2k + c, c
// fixing the parity (bs[3] even, so the sites of one parity alternate along
// x3), positions from nsite/2 on the local-odd sites.  A half pass then runs
// whole warps instead of every other lane.
__device__ __forceinline__ int eo_pos(int n, int par, int half) { return par * half + (n >> 1); }

template <int MU>
__device__ __forceinline__ void sm_block_hop_eo(const SapSm& m, const int bs[4], int n, int par, int half,
                                                const int l[4], Spinor<float>& acc) {
  int stride = 1;
  for (int nu = 3; nu > MU; --nu) stride *= bs[nu];
  const int t = eo_pos(n, par, half);
  if (l[MU] + 1 < bs[MU]) {
    Spinor<float> nb;
    load_smem(m.r, m.nsite, eo_pos(n + stride, par ^ 1, half), nb);
    HalfSpinor<float> h, r;
    project<MU, -1>(nb, h);
    Su3<float> u;
    sm_link(m, MU, t, u);
    su3_mul(u, h, r);
    accum_reconstruct<MU, -1>(acc, r, -0.5f);
  }
  if (l[MU] > 0) {
    const int tb = eo_pos(n - stride, par ^ 1, half);
    Spinor<float> nb;
    load_smem(m.r, m.nsite, tb, nb);
    HalfSpinor<float> h, r;
    project<MU, +1>(nb, h);
    Su3<float> u;
    sm_link(m, MU, tb, u);  // U_mu(x - mu): the forward link of the site below
    su3_dag_mul(u, h, r);
    accum_reconstruct<MU, +1>(acc, r, -0.5f);
  }
}

// acc = D_hop v (in-block hops of the shared field)
__device__ __forceinline__ void sm_dhop(const SapSm& m, const int bs[4], int n, int par, int half, const int l[4],
                                        Spinor<float>& acc) {
  zero_spinor(acc);
  sm_block_hop_eo<0>(m, bs, n, par, half, l, acc);
  sm_block_hop_eo<1>(m, bs, n, par, half, l, acc);
  sm_block_hop_eo<2>(m, bs, n, par, half, l, acc);
  sm_block_hop_eo<3>(m, bs, n, par, half, l, acc);
}

template <int FMT>
__global__ void __launch_bounds__(256) sap_smem_eo_kernel(const SapArgs a) {
  extern __shared__ float4 sm4[];
  const int nsite = a.bs[0] * a.bs[1] * a.bs[2] * a.bs[3];
  SapSm m;
  m.nsite = nsite;
  m.a = sm4;
  m.u = reinterpret_cast<float2*>(sm4 + 18 * nsite);
  m.r = reinterpret_cast<float*>(m.u + 36 * nsite);
  double* red = reinterpret_cast<double*>(m.r + 24 * nsite);
  const int t = threadIdx.x;
  const bool act = t < nsite;
  const int half3 = a.nb[3] / 2;
  int row = blockIdx.x / half3;
  const int mb = blockIdx.x % half3;
  const int bc2 = row % a.nb[2];
  row /= a.nb[2];
  const int bc1 = row % a.nb[1];
  const int bc0 = row / a.nb[1];
  const int bc3 = 2 * mb + ((a.colour + bc0 + bc1 + bc2) & 1);
  // thread t holds the site at parity-sorted position t (see eo_pos)
  const int half = nsite >> 1;
  const int par = (act && t >= half) ? 1 : 0;  // block-local parity
  int l[4], x[4], n;
  {
    const int k = act ? t - par * half : 0;
    int rr = (2 * k) / a.bs[3];  // the row (l0, l1, l2) of in-block index 2k + c
    l[2] = rr % a.bs[2];
    rr /= a.bs[2];
    l[1] = rr % a.bs[1];
    l[0] = rr / a.bs[1];
    const int c = (par + l[0] + l[1] + l[2]) & 1;
    l[3] = (2 * k) % a.bs[3] + c;
    n = 2 * k + c;
  }
  x[0] = bc0 * a.bs[0] + l[0];
  x[1] = bc1 * a.bs[1] + l[1];
  x[2] = bc2 * a.bs[2] + l[2];
  x[3] = bc3 * a.bs[3] + l[3];
  const int p = (x[0] + x[1] + x[2] + x[3]) & 1;  // lattice parity (the Schur complement's)
  const long i = eo_index(a.g, x);
  const bool ev = act && p == 0, od = act && p == 1;

  Spinor<float> r;  // block residual (kept for the odd sites' final solve)
  if (act) {
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      Su3<float> u;
      load_link<float, FMT>(a.links, a.g.Vh, p, mu, i, u);
#pragma unroll
      for (int k = 0; k < 9; ++k) m.u[(mu * 9 + k) * nsite + t] = make_float2(u.m[k / 3][k % 3].re, u.m[k / 3][k % 3].im);
    }
    const float4* q = reinterpret_cast<const float4*>(p ? a.clov_inv : a.clov) + (long)p * 18 * a.g.Vh;
#pragma unroll
    for (int k = 0; k < 18; ++k) m.a[k * nsite + t] = __ldg(q + k * a.g.Vh + i);
    HopArgs ha;
    ha.g = a.g;
    ha.links = a.links;
    const char* nbf = a.phi + (long)(1 - p) * a.half_bytes;
    Spinor<float> acc;
    zero_spinor(acc);
    hop_dir<P_F32, FMT, 0, false>(ha, nbf, p, i, x, acc, -0.5f);
    hop_dir<P_F32, FMT, 1, false>(ha, nbf, p, i, x, acc, -0.5f);
    hop_dir<P_F32, FMT, 2, false>(ha, nbf, p, i, x, acc, -0.5f);
    hop_dir<P_F32, FMT, 3, false>(ha, nbf, p, i, x, acc, -0.5f);
    Spinor<float> ph, aph, rh;
    load_spinor<P_F32>(a.phi + (long)p * a.half_bytes, a.g.Vh, i, ph);
    clover_apply<float>(a.clov, a.g.Vh, p, i, ph, aph);
    load_spinor<P_F32>(a.rho + (long)p * a.half_bytes, a.g.Vh, i, rh);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) r.c[s][c] = rh.c[s][c] - (aph.c[s][c] + acc.c[s][c]);
  }
  __syncthreads();  // the staged links and clover are read by the neighbours below
  // odd sites: w_o = A^{-1} r_o into the shared field
  if (od) {
    Spinor<float> w;
    sm_clover(m, t, r, w);
    store_smem(m.r, nsite, t, w);
  }
  __syncthreads();
  // even sites: rhat_e = r_e - D_eo w_o (written at the even positions, read
  // by no one in this phase)
  Spinor<float> rh;
  zero_spinor(rh);
  if (ev) {
    Spinor<float> acc;
    sm_dhop(m, a.bs, n, par, half, l, acc);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) rh.c[s][c] = r.c[s][c] - acc.c[s][c];
    store_smem(m.r, nsite, t, rh);
  }
  double n0 = 0.0;
  if (a.adaptive) {
    if (ev) n0 = site_norm2(rh);
    n0 = block_sum1(n0, red);
  } else {
    __syncthreads();
  }
  double rn_prev = sqrt(n0);

  Spinor<float> xs;
  zero_spinor(xs);
  int steps = 0;
  for (int k = 1; k <= a.nmr; ++k) {
    // odd half pass: t_o = A^{-1} D_oe rhat_e
    if (od) {
      Spinor<float> acc, w;
      sm_dhop(m, a.bs, n, par, half, l, acc);
      sm_clover(m, t, acc, w);
      store_smem(m.r, nsite, t, w);
    }
    __syncthreads();
    // even half pass: q_e = A rhat_e - D_eo t_o, then <q, rhat>, <q, q>
    Spinor<float> pv;
    float pr_re = 0.f, pr_im = 0.f, pp = 0.f;
    if (ev) {
      Spinor<float> own, acc;
      load_smem(m.r, nsite, t, own);
      sm_clover(m, t, own, pv);
      sm_dhop(m, a.bs, n, par, half, l, acc);
      float ar = 0.f, ai = 0.f, a2 = 0.f;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          pv.c[s][c] = pv.c[s][c] - acc.c[s][c];
          cx<float> q2 = pv.c[s][c], v = own.c[s][c];
          ar += q2.re * v.re + q2.im * v.im;
          ai += q2.re * v.im - q2.im * v.re;
          a2 += q2.re * q2.re + q2.im * q2.im;
        }
      pr_re = ar;
      pr_im = ai;
      pp = a2;
    }
    block_sum3(pr_re, pr_im, pp, red);  // barrier: every read of this step is done
    float om_re = 0.f, om_im = 0.f;
    if (pp > 0.f) {
      om_re = pr_re / pp;
      om_im = pr_im / pp;
    }
    const cx<float> om{om_re, om_im};
    double n1 = 0.0;
    if (ev) {
      Spinor<float> own;
      load_smem(m.r, nsite, t, own);
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          cfma(xs.c[s][c], om, own.c[s][c]);
          own.c[s][c] = own.c[s][c] - om * pv.c[s][c];
        }
      store_smem(m.r, nsite, t, own);
      n1 = site_norm2(own);
    }
    steps = k;
    if (a.adaptive) {
      n1 = block_sum1(n1, red);
      const double rn_new = sqrt(n1);
      if ((k >= 4 && rn_new > (double)a.alpha * rn_prev) || rn_new > rn_prev || rn_new < a.tol) break;
      rn_prev = rn_new;
    } else {
      __syncthreads();  // the odd half pass of the next step reads the even residual
    }
  }
  // delta_e = x_e into the shared field; delta_o = A^{-1} (r_o - D_oe delta_e)
  if (ev) store_smem(m.r, nsite, t, xs);
  __syncthreads();
  if (od) {
    Spinor<float> acc, w;
    sm_dhop(m, a.bs, n, par, half, l, acc);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) w.c[s][c] = r.c[s][c] - acc.c[s][c];
    sm_clover(m, t, w, xs);
  }
  if (act) {
    char* pp = a.phi + (long)p * a.half_bytes;
    Spinor<float> ph;
    load_spinor<P_F32>(pp, a.g.Vh, i, ph);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) ph.c[s][c] = ph.c[s][c] + xs.c[s][c];
    store_spinor<P_F32>(pp, a.g.Vh, i, ph);
  }
  if (a.mr_steps && t == 0) atomicAdd(a.mr_steps, (unsigned)steps);
}

size_t sap_smem_bytes(const int bs[4]) {
  const int nsite = bs[0] * bs[1] * bs[2] * bs[3];
  const int threads = (nsite + 31) / 32 * 32;
  return sizeof(float) * (72 + 72 + 24) * (size_t)nsite + sizeof(double) * 3 * (threads / 32);
}

cudaError_t sap_colour(const Geom& g, const int bs[4], int colour, int fmt, const void* links, const void* clov,
                       const void* clov_inv, const void* rho, void* phi, int nmr, int adaptive, float alpha,
                       double tol, unsigned* mr_steps, int kernel, int eo, cudaStream_t s) {
  SapArgs a;
  a.g = g;
  int nblk = 1;
  for (int mu = 0; mu < 4; ++mu) {
    a.bs[mu] = bs[mu];
    a.nb[mu] = g.L[mu] / bs[mu];
    nblk *= a.nb[mu];
  }
  a.colour = colour;
  a.links = links;
  a.clov = clov;
  a.clov_inv = clov_inv;
  a.rho = (const char*)rho;
  a.phi = (char*)phi;
  a.half_bytes = spinor_half_bytes(g.Vh, P_F32);
  a.nmr = nmr;
  a.adaptive = adaptive;
  a.alpha = alpha;
  a.tol = tol;
  a.mr_steps = mr_steps;
  const int nsite = bs[0] * bs[1] * bs[2] * bs[3];
  const int threads = (nsite + 31) / 32 * 32;
  const size_t smem = sizeof(float) * 24 * nsite + sizeof(double) * 3 * (threads / 32);
  dim3 grid(nblk / 2), block(threads);
  if (eo) {
    // even-odd reduced block solver: shared-memory operands only
    const size_t sm2 = sap_smem_bytes(bs);
    if (sm2 > 227 * 1024 || !clov_inv || bs[3] % 2) return cudaErrorInvalidValue;
    if (fmt == LINK_12) {
      cudaFuncSetAttribute(sap_smem_eo_kernel<LINK_12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
      sap_smem_eo_kernel<LINK_12><<<grid, block, sm2, s>>>(a);
    } else {
      cudaFuncSetAttribute(sap_smem_eo_kernel<LINK_18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
      sap_smem_eo_kernel<LINK_18><<<grid, block, sm2, s>>>(a);
    }
    return cudaGetLastError();
  }
  if (kernel == 0) {
    // operands in shared memory (the default), if they fit
    const size_t sm2 = sap_smem_bytes(bs);
    if (sm2 <= 227 * 1024) {
      if (fmt == LINK_12) {
        cudaFuncSetAttribute(sap_smem_kernel<LINK_12>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
        sap_smem_kernel<LINK_12><<<grid, block, sm2, s>>>(a);
      } else {
        cudaFuncSetAttribute(sap_smem_kernel<LINK_18>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
        sap_smem_kernel<LINK_18><<<grid, block, sm2, s>>>(a);
      }
      return cudaGetLastError();
    }
    kernel = 2;
  }
  if (kernel == 2) {
    if (fmt == LINK_12)
      sap_kernel<LINK_12, 2><<<grid, block, smem, s>>>(a);
    else
      sap_kernel<LINK_18, 2><<<grid, block, smem, s>>>(a);
  } else {
    if (fmt == LINK_12)
      sap_kernel<LINK_12, 1><<<grid, block, smem, s>>>(a);
    else
      sap_kernel<LINK_18, 1><<<grid, block, smem, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace oq
