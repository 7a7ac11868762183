// Gauge-equivariant parallel-transport convolution (PTC) layers: the learned
// preconditioner (not in the paper).  A layer maps C_in spinor fields to
// C_out fields,
//
//   out_c'(x) = sum_{q in paths} sum_c W[q][c'][c] (T_q in_c)(x),
//
// paths q = 0 (identity), 1+2mu (+mu: U_mu(x) in(x+mu)), 2+2mu (-mu:
// U_mu(x-mu)^dag in(x-mu)), with the fermion time-boundary factor on hops
// across the time boundary; W[q][c'][c] is a complex 4x4 matrix on spin.
// Weights are used in bfloat16 (rounded from binary32 master weights),
// arithmetic and accumulation binary32, gradient reductions binary64.
//
// The adjoint of a layer (the backward pass for the input) is again a layer:
// W'[reverse(q)][c][c'] = W[q][c'][c]^dag, since T_{+mu}^dag = T_{-mu}.
// Weight gradients: dW[q][c'][c] = sum_x g_c'(x) (T_q in_c)(x)^dag (spin outer
// product, colour summed): per-CTA binary64 partials, summed in a fixed order.
#include <math.h>
#include <string.h>

#include <vector>

#include "../../include/oq.h"
#include "ctx.h"
#include "oq_kernels.h"
#include "reduce.cuh"

namespace oq {

static const int NPATH = 9;
static const int PB = 128;  // threads per CTA

struct PtcArgs {
  Geom g;
  const void* links;  // binary32 packed links
  const char* in;     // C_in packed binary32 full fields
  char* out;          // C_out packed binary32 full fields
  long fbytes;        // bytes of one full field
  long hbytes;        // bytes of one half field
  const __nv_bfloat162* w;  // [NPATH][C_out][C_in][4][4] complex, bfloat16
};

// (T_q psi)(x) for site (p, i, x) of a full field `f`
template <int FMT>
__device__ __forceinline__ void transport(const PtcArgs& a, const char* f, int q, int p, long i, const int x[4],
                                          Spinor<float>& t) {
  if (q == 0) {
    load_spinor<P_F32>(f + (long)p * a.hbytes, a.g.Vh, i, t);
    return;
  }
  const int mu = (q - 1) >> 1;
  const bool fwd = ((q - 1) & 1) == 0;
  bool cr;
  const long j = eo_neighbour_rt(a.g, x, mu, fwd ? +1 : -1, &cr);
  Spinor<float> s;
  load_spinor<P_F32>(f + (long)(1 - p) * a.hbytes, a.g.Vh, j, s);
  Su3<float> u;
  if (fwd)
    load_link<float, FMT>(a.links, a.g.Vh, p, mu, i, u);
  else
    load_link<float, FMT>(a.links, a.g.Vh, 1 - p, mu, j, u);
  const float sg = cr ? a.g.bc_t : 1.0f;
#pragma unroll
  for (int sp = 0; sp < 4; ++sp)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      cx<float> acc{0.f, 0.f};
#pragma unroll
      for (int b = 0; b < 3; ++b) {
        if (fwd)
          cfma(acc, u.m[c][b], s.c[sp][b]);
        else
          cfmac(acc, u.m[b][c], s.c[sp][b]);
      }
      t.c[sp][c] = sg * acc;
    }
}

template <int FMT, int CIN, int COUT>
__global__ void __launch_bounds__(PB) ptc_layer_kernel(const PtcArgs a) {
  __shared__ float2 w[NPATH * COUT * CIN * 16];
  for (int k = threadIdx.x; k < NPATH * COUT * CIN * 16; k += blockDim.x) w[k] = __bfloat1622float2(a.w[k]);
  __syncthreads();
  const long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 2 * a.g.Vh) return;
  const int p = j >= a.g.Vh ? 1 : 0;
  const long i = j - p * a.g.Vh;
  int x[4];
  eo_coords(a.g, p, i, x);
  Spinor<float> acc[COUT];
#pragma unroll
  for (int co = 0; co < COUT; ++co)
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[co].c[s][c] = cx<float>{0.f, 0.f};
  for (int q = 0; q < NPATH; ++q) {
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) {
      Spinor<float> t;
      transport<FMT>(a, a.in + ci * a.fbytes, q, p, i, x, t);
#pragma unroll
      for (int co = 0; co < COUT; ++co) {
        const float2* ww = w + ((q * COUT + co) * CIN + ci) * 16;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int tt = 0; tt < 4; ++tt) {
            const cx<float> wv{ww[s * 4 + tt].x, ww[s * 4 + tt].y};
#pragma unroll
            for (int c = 0; c < 3; ++c) cfma(acc[co].c[s][c], wv, t.c[tt][c]);
          }
      }
    }
  }
#pragma unroll
  for (int co = 0; co < COUT; ++co) store_spinor<P_F32>(a.out + co * a.fbytes + (long)p * a.hbytes, a.g.Vh, i, acc[co]);
}

// Weight-gradient partials for one path (blockIdx.y): COUT*CIN*16 complex per
// CTA, binary64, written to part[q][cta][k].
template <int FMT, int CIN, int COUT>
__global__ void __launch_bounds__(PB) ptc_dw_kernel(const PtcArgs a, const char* grad, double* part) {
  constexpr int NW = COUT * CIN * 16;  // complex entries per path
  __shared__ double red[PB / 32][2 * NW];
  const int q = blockIdx.y;
  float accr[NW], acci[NW];
#pragma unroll
  for (int k = 0; k < NW; ++k) accr[k] = acci[k] = 0.f;
  for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < 2 * a.g.Vh; j += (long)gridDim.x * blockDim.x) {
    const int p = j >= a.g.Vh ? 1 : 0;
    const long i = j - p * a.g.Vh;
    int x[4];
    eo_coords(a.g, p, i, x);
    Spinor<float> gv[COUT];
#pragma unroll
    for (int co = 0; co < COUT; ++co) load_spinor<P_F32>(grad + co * a.fbytes + (long)p * a.hbytes, a.g.Vh, i, gv[co]);
#pragma unroll
    for (int ci = 0; ci < CIN; ++ci) {
      Spinor<float> t;
      transport<FMT>(a, a.in + ci * a.fbytes, q, p, i, x, t);
#pragma unroll
      for (int co = 0; co < COUT; ++co)
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int tt = 0; tt < 4; ++tt) {
            cx<float> v{0.f, 0.f};
#pragma unroll
            for (int c = 0; c < 3; ++c) cfmac(v, t.c[tt][c], gv[co].c[s][c]);  // g[s] conj(t[t])
            const int k = (co * CIN + ci) * 16 + s * 4 + tt;
            accr[k] += v.re;
            acci[k] += v.im;
          }
    }
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < NW; ++k) {
    double r = warp_sum((double)accr[k]);
    double m = warp_sum((double)acci[k]);
    if (lane == 0) {
      red[wid][2 * k] = r;
      red[wid][2 * k + 1] = m;
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * NW; k += blockDim.x) {
    double s = 0.0;
    for (int w = 0; w < PB / 32; ++w) s += red[w][k];
    part[((long)q * gridDim.x + blockIdx.x) * 2 * NW + k] = s;
  }
}

// sum the per-CTA partials in a fixed order: dw[q][k] += sum_cta part[q][cta][k]
__global__ void ptc_dw_finish(const double* part, int ncta, int nw2, double* dw) {
  const int q = blockIdx.x;
  for (int k = threadIdx.x; k < nw2; k += blockDim.x) {
    double s = 0.0;
    for (int c = 0; c < ncta; ++c) s += part[((long)q * ncta + c) * nw2 + k];
    dw[(long)q * nw2 + k] += s;
  }
}

// bfloat16 forward weights and the adjoint layer's weights from binary32 masters:
// w: [q][co][ci][s][t]; adjoint: [rev(q)][ci][co][t][s] = conj(w[q][co][ci][s][t])
__global__ void ptc_prepare_weights(const float2* master, int cin, int cout, __nv_bfloat162* fwd,
                                    __nv_bfloat162* adj) {
  const int n = NPATH * cout * cin * 16;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    int r = k;
    const int t = r % 4;
    r /= 4;
    const int s = r % 4;
    r /= 4;
    const int ci = r % cin;
    r /= cin;
    const int co = r % cout;
    const int q = r / cout;
    const float2 v = master[k];
    fwd[k] = __floats2bfloat162_rn(v.x, v.y);
    const int qr = q == 0 ? 0 : (((q - 1) & 1) ? q - 1 : q + 1);
    // adjoint layer has C_in' = cout, C_out' = cin
    const int ka = ((qr * cin + ci) * cout + co) * 16 + t * 4 + s;
    adj[ka] = __floats2bfloat162_rn(v.x, -v.y);
  }
}

// g = 2 (y - e) / ||e||^2, loss partial ||y - e||^2 / ||e||^2 -> FIN_STORE slot
__global__ void __launch_bounds__(256) ptc_loss_kernel(const char* y, const char* e, char* g, double inv_en2, long Vh,
                                                       long hb, RedArgs ra) {
  __shared__ double smem[8];
  double acc = 0.0;
  for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < 2 * Vh; j += (long)gridDim.x * blockDim.x) {
    const int p = j >= Vh ? 1 : 0;
    const long i = j - p * Vh;
    Spinor<float> a, b;
    load_spinor<P_F32>(y + p * hb, Vh, i, a);
    load_spinor<P_F32>(e + p * hb, Vh, i, b);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        a.c[s][c] = a.c[s][c] - b.c[s][c];
        acc += (double)a.c[s][c].re * a.c[s][c].re + (double)a.c[s][c].im * a.c[s][c].im;
        a.c[s][c] = (float)(2.0 * inv_en2) * a.c[s][c];
      }
    store_spinor<P_F32>(g + p * hb, Vh, i, a);
  }
  grid_reduce(acc * inv_en2, ra, 0, 1, smem, blockIdx.x, gridDim.x);
}

// Adam on binary32 master weights (per real component), gradient in binary64
__global__ void ptc_adam(float* w, float* m, float* v, const double* g, int n, float lr, float b1, float b2,
                         float c1, float c2, float eps) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const float gk = (float)g[k];
  const float mk = b1 * m[k] + (1.f - b1) * gk;
  const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
  m[k] = mk;
  v[k] = vk;
  w[k] -= lr * (mk / c1) / (sqrtf(vk / c2) + eps);
}

template <int CIN, int COUT>
static cudaError_t ptc_layer(const PtcArgs& a, int fmt, cudaStream_t s) {
  dim3 grid((unsigned)((2 * a.g.Vh + PB - 1) / PB)), block(PB);
  if (fmt == LINK_12)
    ptc_layer_kernel<LINK_12, CIN, COUT><<<grid, block, 0, s>>>(a);
  else
    ptc_layer_kernel<LINK_18, CIN, COUT><<<grid, block, 0, s>>>(a);
  return cudaGetLastError();
}

template <int CIN, int COUT>
static cudaError_t ptc_dw(const PtcArgs& a, int fmt, const char* grad, double* part, int ncta, cudaStream_t s) {
  dim3 grid(ncta, NPATH), block(PB);
  if (fmt == LINK_12)
    ptc_dw_kernel<LINK_12, CIN, COUT><<<grid, block, 0, s>>>(a, grad, part);
  else
    ptc_dw_kernel<LINK_18, CIN, COUT><<<grid, block, 0, s>>>(a, grad, part);
  return cudaGetLastError();
}

}  // namespace oq

using namespace oq;

namespace {
const int CH = 2;                      // hidden feature fields
const int NW1 = NPATH * CH * 1 * 16;   // complex weights of layer 1 (1 -> CH)
const int NW2 = NPATH * 1 * CH * 16;   // complex weights of layer 2 (CH -> 1)

struct NnBufs {
  __nv_bfloat162 *w1, *w2, *w1a, *w2a;
  char* hid;   // CH fields
  char* ghid;  // CH fields
  char* y;
  char* gy;
};

int nn_bufs(oq_handle h, int lat, NnBufs* b) {
  const long f32 = 2 * spinor_half_bytes(h->lats[lat].g.Vh, P_F32);
  void *wb, *hid, *ghid, *y, *gy;
  int rc = 0;
  rc |= h->workspace(lat, "nn_w", sizeof(__nv_bfloat162) * 2 * (NW1 + NW2), &wb);
  rc |= h->workspace(lat, "nn_hid", f32 * CH, &hid);
  rc |= h->workspace(lat, "nn_ghid", f32 * CH, &ghid);
  rc |= h->workspace(lat, "nn_y", f32, &y);
  rc |= h->workspace(lat, "nn_gy", f32, &gy);
  if (rc) return OQ_ERR_NOMEM;
  b->w1 = (__nv_bfloat162*)wb;
  b->w2 = b->w1 + NW1;
  b->w1a = b->w2 + NW2;
  b->w2a = b->w1a + NW1;
  b->hid = (char*)hid;
  b->ghid = (char*)ghid;
  b->y = (char*)y;
  b->gy = (char*)gy;
  return OQ_OK;
}

int nn_prepare(oq_handle h, const float* master, const NnBufs& b, cudaStream_t s) {
  ptc_prepare_weights<<<4, 256, 0, s>>>((const float2*)master, 1, CH, b.w1, b.w1a);
  ptc_prepare_weights<<<4, 256, 0, s>>>((const float2*)master + NW1, CH, 1, b.w2, b.w2a);
  h->launches += 2;
  return cudaGetLastError() == cudaSuccess ? OQ_OK : OQ_ERR_CUDA;
}

PtcArgs nn_args(oq_handle h, int lat) {
  const LatCtx& L = h->lats[lat];
  PtcArgs a;
  a.g = L.g;
  a.links = L.u32.p;
  a.hbytes = spinor_half_bytes(L.g.Vh, P_F32);
  a.fbytes = 2 * a.hbytes;
  return a;
}

// y = L2(L1(r)) with the prepared bfloat16 weights
int nn_forward(oq_handle h, int lat, const NnBufs& b, const void* r, void* y, cudaStream_t s) {
  const int fmt = h->lats[lat].link_fmt;
  PtcArgs a = nn_args(h, lat);
  a.in = (const char*)r;
  a.out = b.hid;
  a.w = b.w1;
  if (ptc_layer<1, CH>(a, fmt, s) != cudaSuccess) return OQ_ERR_CUDA;
  a.in = b.hid;
  a.out = (char*)y;
  a.w = b.w2;
  if (ptc_layer<CH, 1>(a, fmt, s) != cudaSuccess) return OQ_ERR_CUDA;
  h->launches += 2;
  return OQ_OK;
}

}  // namespace

// internal: the learned preconditioner as used inside flexible GCR
namespace oq {
int nnprec_prepare(oq_handle h, int lat, const float* master, cudaStream_t s) {
  NnBufs b;
  int rc = nn_bufs(h, lat, &b);
  if (rc) return rc;
  return nn_prepare(h, master, b, s);
}
int nnprec_forward(oq_handle h, int lat, const void* r, void* y, cudaStream_t s) {
  NnBufs b;
  int rc = nn_bufs(h, lat, &b);
  if (rc) return rc;
  return nn_forward(h, lat, b, r, y, s);
}
}  // namespace oq

extern "C" int oq_nnprec_apply(oq_handle h, int lat, const float* weights_dev, const void* in_dev, void* out_dev,
                               void* stream) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || !weights_dev || !in_dev || !out_dev) return OQ_ERR_ARG;
  if (!h->lats[lat].has_gauge || h->lats[lat].halo_t) return OQ_ERR_STATE;  // whole lattices only
  cudaStream_t s = (cudaStream_t)stream;
  int rc = nnprec_prepare(h, lat, weights_dev, s);
  if (rc) return rc;
  return nnprec_forward(h, lat, in_dev, out_dev, s);
}

extern "C" int oq_nnprec_grad(oq_handle h, int lat, const float* weights_dev, const void* r_dev, const void* e_dev,
                              int n, double* grad_dev, double* loss_host, void* stream);

extern "C" int oq_nnprec_train(oq_handle h, int lat, float* weights_dev, const void* r_dev, const void* e_dev, int n,
                               double lr, int steps, double* loss_host, void* stream) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || !weights_dev || !r_dev || !e_dev || n < 1 || steps < 1 ||
      !(lr > 0.0))
    return OQ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int nreal = 2 * (NW1 + NW2);
  void *mom, *grad;
  int rc = h->workspace(lat, "nn_adam", sizeof(float) * 2 * nreal, &mom);
  if (!rc) rc = h->workspace(lat, "nn_gradbuf", sizeof(double) * nreal, &grad);
  if (rc) return OQ_ERR_NOMEM;
  if (cudaMemsetAsync(mom, 0, sizeof(float) * 2 * nreal, s) != cudaSuccess) return OQ_ERR_CUDA;
  const float b1 = 0.9f, b2 = 0.999f;
  float p1 = 1.f, p2 = 1.f;
  for (int it = 0; it < steps; ++it) {
    double loss = 0.0;
    rc = oq_nnprec_grad(h, lat, weights_dev, r_dev, e_dev, n, (double*)grad, &loss, stream);
    if (rc) return rc;
    if (loss_host) loss_host[it] = loss;
    p1 *= b1;
    p2 *= b2;
    ptc_adam<<<(nreal + 255) / 256, 256, 0, s>>>(weights_dev, (float*)mom, (float*)mom + nreal, (const double*)grad,
                                                 nreal, (float)lr, b1, b2, 1.f - p1, 1.f - p2, 1e-8f);
    h->launches += 1;
    if (cudaGetLastError() != cudaSuccess) return OQ_ERR_CUDA;
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) return OQ_ERR_CUDA;
  return OQ_OK;
}

extern "C" int oq_nnprec_grad(oq_handle h, int lat, const float* weights_dev, const void* r_dev, const void* e_dev,
                              int n, double* grad_dev, double* loss_host, void* stream) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || !weights_dev || !r_dev || !e_dev || n < 1 || !grad_dev)
    return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.has_gauge || L.halo_t) return OQ_ERR_STATE;  // whole lattices only
  cudaStream_t s = (cudaStream_t)stream;
  NnBufs b;
  int rc = nn_bufs(h, lat, &b);
  if (rc) return rc;
  rc = nn_prepare(h, weights_dev, b, s);
  if (rc) return rc;
  const long Vh = L.g.Vh;
  const long hb = spinor_half_bytes(Vh, P_F32), f32 = 2 * hb;
  const int ncta = reduce_grid(2 * Vh) < 256 ? reduce_grid(2 * Vh) : 256;
  void* part;
  rc = h->workspace(lat, "nn_part", sizeof(double) * NPATH * ncta * 2 * 32, &part);
  if (!rc) rc = h->ensure_reduce(2, reduce_grid(2 * Vh));
  if (rc) return rc;
  const int fmt = L.link_fmt;
  const int nreal = 2 * (NW1 + NW2);
  if (cudaMemsetAsync(grad_dev, 0, sizeof(double) * nreal, s) != cudaSuccess) return OQ_ERR_CUDA;
  double* gw1 = grad_dev;
  double* gw2 = grad_dev + 2 * NW1;
  double loss = 0.0;
  for (int k = 0; k < n; ++k) {
    const char* r = (const char*)r_dev + (long)k * f32;
    const char* e = (const char*)e_dev + (long)k * f32;
    // ||e||^2
    RedArgs ra = h->red_args(FIN_STORE, 0);
    h->launches += 2;
    if (reduce_norm2(P_F32, e, Vh, 0, 1, ra, s) != cudaSuccess) return OQ_ERR_CUDA;
    ra.result = h->results + 1;
    if (reduce_norm2(P_F32, e + hb, Vh, 0, 1, ra, s) != cudaSuccess) return OQ_ERR_CUDA;
    if (cudaMemcpyAsync(h->results_host, h->results, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return OQ_ERR_CUDA;
    const double en2 = h->results_host[0] + h->results_host[1];
    if (!(en2 > 0.0)) return OQ_ERR_ARG;
    rc = nn_forward(h, lat, b, r, b.y, s);
    if (rc) return rc;
    ra = h->red_args(FIN_STORE, 0);
    // mean over the n pairs: loss_k / n and its gradient
    ptc_loss_kernel<<<reduce_grid(2 * Vh), 256, 0, s>>>(b.y, e, b.gy, 1.0 / (en2 * n), Vh, hb, ra);
    h->launches += 1;
    if (cudaMemcpyAsync(h->results_host, h->results, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return OQ_ERR_CUDA;
    loss += h->results_host[0];
    // layer 2: dW2 from (hid, gy); g_hid = L2^dag gy
    PtcArgs a = nn_args(h, lat);
    a.in = b.hid;
    a.w = b.w2;
    if (ptc_dw<CH, 1>(a, fmt, b.gy, (double*)part, ncta, s) != cudaSuccess) return OQ_ERR_CUDA;
    ptc_dw_finish<<<NPATH, 128, 0, s>>>((const double*)part, ncta, 2 * CH * 16, gw2);
    a.in = b.gy;
    a.out = b.ghid;
    a.w = b.w2a;
    if (ptc_layer<1, CH>(a, fmt, s) != cudaSuccess) return OQ_ERR_CUDA;
    // layer 1: dW1 from (r, g_hid)
    a = nn_args(h, lat);
    a.in = r;
    a.w = b.w1;
    if (ptc_dw<1, CH>(a, fmt, b.ghid, (double*)part, ncta, s) != cudaSuccess) return OQ_ERR_CUDA;
    ptc_dw_finish<<<NPATH, 128, 0, s>>>((const double*)part, ncta, 2 * CH * 16, gw1);
    h->launches += 5;
    if (cudaGetLastError() != cudaSuccess) return OQ_ERR_CUDA;
  }
  if (loss_host) *loss_host = loss;
  return OQ_OK;
}
