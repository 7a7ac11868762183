// Flexible GCR with restarts and the SAP preconditioner (Sec. 3.1, Table 2):
// solves D psi = eta on the full lattice.
//
// Per step k < nkv:   phi_k = M rho_k        (SAP cycles, or identity if ncy = 0)
//                     chi_k = D phi_k
//                     a_lk = <chi_l, chi_k>, chi_k -= sum_l a_lk chi_l (classical
//                     Gram-Schmidt: all dots in one launch, one fused update)
//                     b_k = ||chi_k||, chi_k /= b_k, c_k = <chi_k, rho_k>,
//                     rho_{k+1} = rho_k - c_k chi_k
// Restart / finish:   b_l beta_l + sum_{m>l} a_lm beta_m = c_l (host, k <= nkv),
//                     psi += sum_l beta_l phi_l (binary64), rho = eta - D psi
//                     (binary64 stencil: the "large" type).
// The Krylov vectors, SAP and the regular steps use binary32 (the "small"
// type); every reduction is binary64 (the reduction type).
#include <math.h>
#include <string.h>

#include <complex>
#include <vector>

#include "../../include/oq.h"
#include "ctx.h"
#include "oq_kernels.h"
#include "reduce.cuh"

namespace oq {

static const int VB = 256;

// site j of a full field (two half fields of Vh sites)
__device__ __forceinline__ const char* fsite(const char* base, long Vh, long half_bytes, long j, long* i) {
  const long h = j >= Vh ? 1 : 0;
  *i = j - h * Vh;
  return base + h * half_bytes;
}

// <a, b> of one site added to (re, im).  Binary32 fields (the GCR Krylov
// vectors): the site's 12 complex terms summed in binary32 by FMAs, the sums
// over sites in binary64 -- binary64 arithmetic runs at 1/64 of the binary32
// rate on GB300, and widening every term had made these dots FP64-bound.
// Binary64 fields: binary64 throughout.
template <typename R>
__device__ __forceinline__ void site_dot(const Spinor<R>& a, const Spinor<R>& b, double& re, double& im) {
  if constexpr (std::is_same<R, float>::value) {
    float sr = 0.f, si = 0.f;
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        sr = fmaf(a.c[s][c].re, b.c[s][c].re, fmaf(a.c[s][c].im, b.c[s][c].im, sr));
        si = fmaf(a.c[s][c].re, b.c[s][c].im, fmaf(-a.c[s][c].im, b.c[s][c].re, si));
      }
    re += (double)sr;
    im += (double)si;
  } else {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        re += (double)a.c[s][c].re * b.c[s][c].re + (double)a.c[s][c].im * b.c[s][c].im;
        im += (double)a.c[s][c].re * b.c[s][c].im - (double)a.c[s][c].im * b.c[s][c].re;
      }
  }
}

template <int P>
__global__ void __launch_bounds__(VB) vec_dots_kernel(const char* X, long xstride, const char* y, long Vh,
                                                      long hb, RedArgs ra, int nl) {
  typedef typename PrecTraits<P>::R R;
  __shared__ double smem[VB / 32];
  const int l = blockIdx.y;
  double re = 0.0, im = 0.0;
  for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < 2 * Vh; j += (long)gridDim.x * blockDim.x) {
    long i;
    Spinor<R> a, b;
    load_spinor<P>(fsite(X + l * xstride, Vh, hb, j, &i), Vh, i, a);
    load_spinor<P>(fsite(y, Vh, hb, j, &i), Vh, i, b);
    site_dot(a, b, re, im);
  }
  grid_reduce(re, ra, 2 * l, 2 * nl, smem, blockIdx.x, gridDim.x);
  __syncthreads();
  grid_reduce(im, ra, 2 * l + 1, 2 * nl, smem, blockIdx.x, gridDim.x);
}

// chi -= sum_l coef_l X_l ; ||chi||^2 -> slot 0
template <int P>
__global__ void __launch_bounds__(VB) vec_orth_kernel(char* chi, const char* X, long xstride,
                                                      const double2* coef, int nl, long Vh, long hb, RedArgs ra) {
  typedef typename PrecTraits<P>::R R;
  __shared__ double smem[VB / 32];
  double acc = 0.0;
  for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < 2 * Vh; j += (long)gridDim.x * blockDim.x) {
    long i;
    char* cb = (char*)fsite(chi, Vh, hb, j, &i);
    Spinor<R> v;
    load_spinor<P>(cb, Vh, i, v);
    for (int l = 0; l < nl; ++l) {
      Spinor<R> w;
      load_spinor<P>(fsite(X + l * xstride, Vh, hb, j, &i), Vh, i, w);
      const cx<R> c{(R)coef[l].x, (R)coef[l].y};
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) v.c[s][a] = v.c[s][a] - c * w.c[s][a];
    }
    store_spinor<P>(cb, Vh, i, v);
    acc += site_norm2(v);
  }
  grid_reduce(acc, ra, 0, 1, smem, blockIdx.x, gridDim.x);
}

// chi *= inv_b ; <chi, rho> -> slots 0, 1
template <int P>
__global__ void __launch_bounds__(VB) vec_scale_dot_kernel(char* chi, const char* rho, double inv_b, long Vh,
                                                           long hb, RedArgs ra) {
  typedef typename PrecTraits<P>::R R;
  __shared__ double smem[VB / 32];
  double re = 0.0, im = 0.0;
  for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < 2 * Vh; j += (long)gridDim.x * blockDim.x) {
    long i;
    char* cb = (char*)fsite(chi, Vh, hb, j, &i);
    Spinor<R> v, r;
    load_spinor<P>(cb, Vh, i, v);
    load_spinor<P>(fsite(rho, Vh, hb, j, &i), Vh, i, r);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) v.c[s][a] = (R)inv_b * v.c[s][a];
    site_dot(v, r, re, im);
    store_spinor<P>(cb, Vh, i, v);
  }
  grid_reduce(re, ra, 0, 2, smem, blockIdx.x, gridDim.x);
  __syncthreads();
  grid_reduce(im, ra, 1, 2, smem, blockIdx.x, gridDim.x);
}

// rho -= c chi ; ||rho||^2 -> slot 0
template <int P>
__global__ void __launch_bounds__(VB) vec_axpy_norm_kernel(char* rho, const char* chi, double cre, double cim,
                                                           long Vh, long hb, RedArgs ra) {
  typedef typename PrecTraits<P>::R R;
  __shared__ double smem[VB / 32];
  double acc = 0.0;
  const cx<R> c{(R)cre, (R)cim};
  for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < 2 * Vh; j += (long)gridDim.x * blockDim.x) {
    long i;
    char* rb = (char*)fsite(rho, Vh, hb, j, &i);
    Spinor<R> v, w;
    load_spinor<P>(rb, Vh, i, v);
    load_spinor<P>(fsite(chi, Vh, hb, j, &i), Vh, i, w);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) v.c[s][a] = v.c[s][a] - c * w.c[s][a];
    store_spinor<P>(rb, Vh, i, v);
    acc += site_norm2(v);
  }
  grid_reduce(acc, ra, 0, 1, smem, blockIdx.x, gridDim.x);
}

// out = a - b (out may be null: norm only) ; ||a - b||^2 -> slot 0 (binary64 products)
template <int P>
__global__ void __launch_bounds__(VB) vec_diff_norm_kernel(char* out, const char* a, const char* b, long Vh,
                                                           long hb, RedArgs ra) {
  typedef typename PrecTraits<P>::R R;
  __shared__ double smem[VB / 32];
  double acc = 0.0;
  for (long j = (long)blockIdx.x * blockDim.x + threadIdx.x; j < 2 * Vh; j += (long)gridDim.x * blockDim.x) {
    long i;
    Spinor<R> v, w;
    load_spinor<P>(fsite(a, Vh, hb, j, &i), Vh, i, v);
    load_spinor<P>(fsite(b, Vh, hb, j, &i), Vh, i, w);
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        v.c[s][c] = v.c[s][c] - w.c[s][c];
        acc += (double)v.c[s][c].re * v.c[s][c].re + (double)v.c[s][c].im * v.c[s][c].im;
      }
    if (out) store_spinor<P>((char*)fsite(out, Vh, hb, j, &i), Vh, i, v);
  }
  grid_reduce(acc, ra, 0, 1, smem, blockIdx.x, gridDim.x);
}

// out (PO) = in (PI), full fields
template <int PI, int PO>
__global__ void __launch_bounds__(VB) vec_convert_kernel(char* out, const char* in, long Vh, long hbi, long hbo) {
  typedef typename PrecTraits<PI>::R RI;
  typedef typename PrecTraits<PO>::R RO;
  const long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 2 * Vh) return;
  long i;
  Spinor<RI> v;
  load_spinor<PI>(fsite(in, Vh, hbi, j, &i), Vh, i, v);
  Spinor<RO> w;
#pragma unroll
  for (int s = 0; s < 4; ++s)
#pragma unroll
    for (int c = 0; c < 3; ++c) w.c[s][c] = cx<RO>{(RO)v.c[s][c].re, (RO)v.c[s][c].im};
  store_spinor<PO>((char*)fsite(out, Vh, hbo, j, &i), Vh, i, w);
}

// psi (F64) += sum_l beta_l Phi_l (F32)
__global__ void __launch_bounds__(VB) vec_psi_update_kernel(char* psi, const char* Phi, long pstride,
                                                            const double2* beta, int nl, long Vh, long hb64,
                                                            long hb32) {
  const long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= 2 * Vh) return;
  long i;
  char* pb = (char*)fsite(psi, Vh, hb64, j, &i);
  Spinor<double> v;
  load_spinor<P_F64>(pb, Vh, i, v);
  for (int l = 0; l < nl; ++l) {
    Spinor<float> w;
    load_spinor<P_F32>(fsite(Phi + l * pstride, Vh, hb32, j, &i), Vh, i, w);
    const cx<double> c{beta[l].x, beta[l].y};
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
      for (int a = 0; a < 3; ++a) v.c[s][a] = v.c[s][a] + c * cx<double>{(double)w.c[s][a].re, (double)w.c[s][a].im};
  }
  store_spinor<P_F64>(pb, Vh, i, v);
}

}  // namespace oq

using namespace oq;

extern "C" int oq_sap_apply(oq_handle h, int lat, const oq_solver_params* prm, const void* rho_dev, void* phi_dev,
                            double mr_tol, void* stream) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || !prm || !rho_dev || !phi_dev || prm->ncy < 1 || prm->nmr < 0 ||
      (prm->sap_eo != 0 && prm->sap_eo != 1) || (prm->sap_eo && prm->bs[3] % 2))
    return OQ_ERR_ARG;
  LatCtx& L = h->lats[lat];
  if (!L.has_clover || L.halo_t) return OQ_ERR_STATE;  // whole lattices only
  int bvol = 1;
  for (int mu = 0; mu < 4; ++mu) {
    const int b = prm->bs[mu];
    if (b < 1 || L.g.L[mu] % b || (L.g.L[mu] / b) % 2) return OQ_ERR_ARG;
    bvol *= b;
  }
  if (bvol > 256) return OQ_ERR_ARG;
  // shifted (C*) wraps keep the block colouring only if the x1 shift is an even number of blocks
  if (L.g.cs_shift && ((L.g.L[1] / 2) / prm->bs[1]) % 2) return OQ_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const long f32 = 2 * spinor_half_bytes(L.g.Vh, P_F32);
  if (cudaMemsetAsync(phi_dev, 0, f32, s) != cudaSuccess) return OQ_ERR_CUDA;
  const float alpha = (float)(prm->alpha > 0.0 ? prm->alpha : 0.9);
  for (int cy = 0; cy < prm->ncy; ++cy)
    for (int colour = 0; colour < 2; ++colour) {
      h->launches += 1;
      if (sap_colour(L.g, prm->bs, colour, L.link_fmt, L.u32.p, L.a32.p, L.i32.p, rho_dev, phi_dev, prm->nmr,
                     prm->adaptive, alpha, mr_tol, nullptr, h->sap_kernel, prm->sap_eo, s) != cudaSuccess)
        return OQ_ERR_CUDA;
    }
  return OQ_OK;
}

static int gcr_impl(oq_handle h, int lat, const oq_solver_params* prm, const float* nn_w, const double* eta_dev,
                    double* psi_dev, int nrhs, oq_status* st, void* stream);

extern "C" int oq_sap_gcr_solve(oq_handle h, int lat, const oq_solver_params* prm, const double* eta_dev,
                                double* psi_dev, int nrhs, oq_status* st, void* stream) {
  return gcr_impl(h, lat, prm, nullptr, eta_dev, psi_dev, nrhs, st, stream);
}

extern "C" int oq_nn_gcr_solve(oq_handle h, int lat, const oq_solver_params* prm, const float* weights_dev,
                               const double* eta_dev, double* psi_dev, int nrhs, oq_status* st, void* stream) {
  if (!weights_dev) return OQ_ERR_ARG;
  return gcr_impl(h, lat, prm, weights_dev, eta_dev, psi_dev, nrhs, st, stream);
}

static int gcr_impl(oq_handle h, int lat, const oq_solver_params* prm, const float* nn_w, const double* eta_dev,
                    double* psi_dev, int nrhs, oq_status* st, void* stream) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || !prm || !eta_dev || !psi_dev || nrhs < 1 || !st) return OQ_ERR_ARG;
  if (!(prm->res > 0.0) || prm->nmx < 1 || prm->nkv < 1 || prm->nkv > 64 || prm->ncy < 0 || prm->nmr < 0 ||
      (prm->sap_eo != 0 && prm->sap_eo != 1) || (prm->sap_eo && prm->ncy > 0 && prm->bs[3] % 2))
    return OQ_ERR_ARG;
  if (prm->sdtype != OQ_F32) return OQ_ERR_ARG;  // SAP and the Krylov vectors run in binary32
  LatCtx& L = h->lats[lat];
  if (!L.has_clover || L.halo_t) return OQ_ERR_STATE;  // whole lattices only
  int nblk = 1, bvol = 1;
  if (prm->ncy > 0) {
    for (int mu = 0; mu < 4; ++mu) {
      const int b = prm->bs[mu];
      if (b < 1 || L.g.L[mu] % b || (L.g.L[mu] / b) % 2) return OQ_ERR_ARG;
      nblk *= L.g.L[mu] / b;
      bvol *= b;
    }
    if (bvol > 256) return OQ_ERR_ARG;
    // shifted (C*) wraps keep the block colouring only if the x1 shift is an even number of blocks
    if (L.g.cs_shift && ((L.g.L[1] / 2) / prm->bs[1]) % 2) return OQ_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const long Vh = L.g.Vh;
  const long hb64 = spinor_half_bytes(Vh, P_F64), hb32 = spinor_half_bytes(Vh, P_F32);
  const long f64 = 2 * hb64, f32 = 2 * hb32;
  const int nkv = prm->nkv;
  void *eta64, *psi64, *rho64, *tmp64, *rho, *tmp32, *Phi, *Chi, *coef;
  int rc = 0;
  rc |= h->workspace(lat, "gcr_eta64", f64, &eta64);
  rc |= h->workspace(lat, "gcr_psi64", f64, &psi64);
  rc |= h->workspace(lat, "gcr_rho64", f64, &rho64);
  rc |= h->workspace(lat, "gcr_tmp64", f64, &tmp64);
  rc |= h->workspace(lat, "gcr_rho", f32, &rho);
  rc |= h->workspace(lat, "gcr_tmp32", f32, &tmp32);
  rc |= h->workspace(lat, "gcr_phi", f32 * nkv, &Phi);
  rc |= h->workspace(lat, "gcr_chi", f32 * nkv, &Chi);
  rc |= h->workspace(lat, "gcr_coef", sizeof(double2) * 64, &coef);
  void* mrc = nullptr;
  rc |= h->workspace(lat, "gcr_mrsteps", sizeof(unsigned) * 4, &mrc);
  if (rc) return OQ_ERR_NOMEM;
  if (nn_w) {
    rc = nnprec_prepare(h, lat, nn_w, (cudaStream_t)stream);
    if (rc) return rc;
  }
  const int grid = reduce_grid(2 * Vh);
  rc = h->ensure_reduce(2 * 64, grid);
  if (rc) return rc;
  rc = h->ensure_stage();
  if (rc) return rc;
  double2* coef_host = reinterpret_cast<double2*>(h->stage_host);  // pinned staging of 64 coefficients
  std::vector<double2> cbuf(64);

#define CK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) return OQ_ERR_CUDA; \
  } while (0)
#define KL(x)                                   \
  do {                                          \
    h->launches += 1;                           \
    if ((x) != cudaSuccess) return OQ_ERR_CUDA; \
  } while (0)
#define RK(x)            \
  do {                   \
    int rc_ = (x);       \
    if (rc_) return rc_; \
  } while (0)

  const dim3 rgrid(grid), rblock(VB);
  const dim3 egrid((unsigned)((2 * Vh + VB - 1) / VB)), eblock(VB);
  RedArgs ra = h->red_args(FIN_STORE, 0);
  // read `n` reduction results (synchronises)
  auto fetch = [&](int n, double* out) -> int {
    CK(cudaMemcpyAsync(h->results_host, h->results, sizeof(double) * n, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    for (int k = 0; k < n; ++k) out[k] = h->results_host[k];
    return OQ_OK;
  };
  auto dw = [&](int prec, const void* in, void* out) -> int {
    HopArgs a = h->hop_args(lat, prec);
    a.in = a.in2 = in;
    a.out = out;
    a.nrhs = 1;
    a.half_bytes = prec == P_F64 ? hb64 : hb32;
    a.in_stride = a.in2_stride = a.out_stride = 2 * a.half_bytes;
    return h->run_hop(h->hop_launch(lat, prec, HOP_DW, 0, EPI_NONE, 1), a, s);
  };

  int ret = OQ_OK;
  for (int r = 0; r < nrhs; ++r) {
    const double* eta_r = eta_dev + (long)r * 2 * Vh * 24;
    double* psi_r = psi_dev + (long)r * 2 * Vh * 24;
    KL(pack_spinor(L.g, P_F64, OQ_FULL, eta_r, eta64, 1.0, 1, 2 * Vh * 12, f64, s));
    CK(cudaMemsetAsync(psi64, 0, f64, s));
    CK(cudaMemcpyAsync(rho64, eta64, f64, cudaMemcpyDeviceToDevice, s));
    KL(reduce_norm2(P_F64, eta64, Vh, 0, 1, ra, s));
    KL(reduce_norm2(P_F64, (const char*)eta64 + hb64, Vh, 0, 1, (ra.result = h->results + 1, ra), s));
    ra.result = h->results;
    double en2[2];
    RK(fetch(2, en2));
    const double eta_n = sqrt(en2[0] + en2[1]);
    double rn = eta_n;
    const double tol = prm->res * eta_n;
    int status = 0, restarts = 0, cycles_total = 0, precs = 0;
    CK(cudaMemsetAsync(mrc, 0, sizeof(unsigned), s));
    bool nonfinite = false;
    // the learned preconditioner, until a restart cycle fails to halve the
    // binary64 residual: then SAP (ncy > 0) or none takes over for the rest
    // of the solve
    bool use_nn = nn_w != nullptr;
    int fallback = 0;
    while (rn > tol && status < prm->nmx && !nonfinite && eta_n > 0.0) {
      KL((vec_convert_kernel<P_F64, P_F32><<<egrid, eblock, 0, s>>>((char*)rho, (const char*)rho64, Vh, hb64,
                                                                     hb32),
          cudaGetLastError()));
      std::vector<std::complex<double>> a((size_t)nkv * nkv), c(nkv);
      std::vector<double> b(nkv);
      int k_used = 0;
      for (int k = 0; k < nkv; ++k) {
        char* phik = (char*)Phi + (long)k * f32;
        char* chik = (char*)Chi + (long)k * f32;
        // phi_k = M rho
        if (use_nn) {
          if (h->nn_tensor_cores)
            RK(nnprec_forward_tc(h, lat, nn_w, rho, phik, s));
          else
            RK(nnprec_forward(h, lat, rho, phik, s));
          precs += 1;
        } else if (prm->ncy == 0) {
          CK(cudaMemcpyAsync(phik, rho, f32, cudaMemcpyDeviceToDevice, s));
        } else {
          CK(cudaMemsetAsync(phik, 0, f32, s));
          double prev = 0.0;
          if (prm->adaptive) {
            KL((vec_diff_norm_kernel<P_F32><<<rgrid, rblock, 0, s>>>(nullptr, (const char*)rho, (const char*)phik,
                                                                     Vh, hb32, ra),
                cudaGetLastError()));
            RK(fetch(1, &prev));
          }
          for (int cy = 0; cy < prm->ncy; ++cy) {
            for (int colour = 0; colour < 2; ++colour)
              KL(sap_colour(L.g, prm->bs, colour, L.link_fmt, L.u32.p, L.a32.p, L.i32.p, rho, phik, prm->nmr,
                            prm->adaptive, (float)(prm->alpha > 0.0 ? prm->alpha : 0.9), prm->res * eta_n / nblk,
                            (unsigned*)mrc, h->sap_kernel, prm->sap_eo, s));
            cycles_total += 1;
            if (prm->adaptive) {
              // cycle test on the global SAP residual ||rho - D phi||
              RK(dw(P_F32, phik, tmp32));
              KL((vec_diff_norm_kernel<P_F32><<<rgrid, rblock, 0, s>>>(nullptr, (const char*)rho,
                                                                       (const char*)tmp32, Vh, hb32, ra),
                  cudaGetLastError()));
              double now = 0.0;
              RK(fetch(1, &now));
              if (!(now < prev)) break;
              prev = now;
            }
          }
          precs += 1;
        }
        // chi_k = D phi_k
        RK(dw(P_F32, phik, chik));
        double bk2 = 0.0;
        if (k > 0) {
          KL((vec_dots_kernel<P_F32><<<dim3(grid, k), rblock, 0, s>>>((const char*)Chi, f32, chik, Vh, hb32, ra, k),
              cudaGetLastError()));
          std::vector<double> d(2 * k);
          RK(fetch(2 * k, d.data()));
          for (int l = 0; l < k; ++l) {
            a[(size_t)l * nkv + k] = std::complex<double>(d[2 * l], d[2 * l + 1]);
            cbuf[l] = make_double2(d[2 * l], d[2 * l + 1]);
            coef_host[l] = cbuf[l];
          }
          CK(cudaMemcpyAsync(coef, coef_host, sizeof(double2) * k, cudaMemcpyHostToDevice, s));
          KL((vec_orth_kernel<P_F32><<<rgrid, rblock, 0, s>>>(chik, (const char*)Chi, f32, (const double2*)coef, k,
                                                              Vh, hb32, ra),
              cudaGetLastError()));
          RK(fetch(1, &bk2));
        } else {
          KL(reduce_norm2(P_F32, chik, Vh, 0, 1, ra, s));
          KL(reduce_norm2(P_F32, chik + hb32, Vh, 0, 1, (ra.result = h->results + 1, ra), s));
          ra.result = h->results;
          double t2[2];
          RK(fetch(2, t2));
          bk2 = t2[0] + t2[1];
        }
        b[k] = sqrt(bk2);
        if (!(b[k] > 0.0) || !isfinite(b[k])) {
          nonfinite = !isfinite(b[k]);
          k_used = k;
          break;
        }
        KL((vec_scale_dot_kernel<P_F32><<<rgrid, rblock, 0, s>>>(chik, (const char*)rho, 1.0 / b[k], Vh, hb32, ra),
            cudaGetLastError()));
        double cd[2];
        RK(fetch(2, cd));
        c[k] = std::complex<double>(cd[0], cd[1]);
        KL((vec_axpy_norm_kernel<P_F32><<<rgrid, rblock, 0, s>>>((char*)rho, chik, cd[0], cd[1], Vh, hb32, ra),
            cudaGetLastError()));
        double r2 = 0.0;
        RK(fetch(1, &r2));
        status += 1;
        k_used = k + 1;
        if (!isfinite(r2)) {
          nonfinite = true;
          break;
        }
        if (sqrt(r2) <= tol || status >= prm->nmx) break;
      }
      if (k_used == 0) break;
      // back substitution and binary64 update of psi
      std::vector<std::complex<double>> beta(k_used);
      for (int l = k_used - 1; l >= 0; --l) {
        std::complex<double> sum = c[l];
        for (int m = l + 1; m < k_used; ++m) sum -= a[(size_t)l * nkv + m] * beta[m];
        beta[l] = sum / b[l];
      }
      for (int l = 0; l < k_used; ++l) coef_host[l] = make_double2(beta[l].real(), beta[l].imag());
      CK(cudaMemcpyAsync(coef, coef_host, sizeof(double2) * k_used, cudaMemcpyHostToDevice, s));
      KL((vec_psi_update_kernel<<<egrid, eblock, 0, s>>>((char*)psi64, (const char*)Phi, f32, (const double2*)coef,
                                                          k_used, Vh, hb64, hb32),
          cudaGetLastError()));
      // rho = eta - D psi in binary64
      RK(dw(P_F64, psi64, tmp64));
      KL((vec_diff_norm_kernel<P_F64><<<rgrid, rblock, 0, s>>>((char*)rho64, (const char*)eta64, (const char*)tmp64,
                                                               Vh, hb64, ra),
          cudaGetLastError()));
      double r2 = 0.0;
      RK(fetch(1, &r2));
      const double rn_cycle = rn;
      rn = sqrt(r2);
      if (!isfinite(r2)) nonfinite = true;
      restarts += 1;
      if (use_nn && !(rn <= 0.5 * rn_cycle)) {
        use_nn = false;
        fallback = 1;
      }
    }
    unsigned mr_total = 0;
    CK(cudaMemcpyAsync(&mr_total, mrc, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    CK(cudaMemsetAsync(psi_r, 0, sizeof(double) * 2 * Vh * 24, s));
    KL(unpack_spinor(L.g, P_F64, OQ_FULL, psi64, psi_r, 1.0, 1, f64, 2 * Vh * 12, s));
    CK(cudaStreamSynchronize(s));
    st[r].steps = status;
    st[r].resets = 0;
    st[r].restarts = restarts;
    st[r].true_rel_res = eta_n > 0.0 ? rn / eta_n : 0.0;
    st[r].converged = (!nonfinite && rn <= tol) ? 1 : 0;
    st[r].cycles = cycles_total;
    st[r].nn_fallback = fallback;
    st[r].mr_avg = (precs > 0 && cycles_total > 0 && nblk > 0) ? (double)mr_total / ((double)cycles_total * nblk)
                                                              : 0.0;
    for (int i = 0; i < 4; ++i) st[r].ladder_steps[i] = 0;
    if (nonfinite) ret = OQ_ERR_NONFINITE;
    else if (!st[r].converged && ret == OQ_OK) ret = OQ_ERR_NOCONV;
  }
  return ret;
#undef CK
#undef KL
#undef RK
}
