// Batched CGNE with reset steps over an uneven batch of systems (lattices of
// different sizes or operators, one right-hand side each), for many small
// and medium lattices at once (QCD+QED: several charges and volumes).
//
// Same algorithm as oq_cgne_solve (Sec. 2), organised for launch overhead:
//  * every stencil pass of every system is ONE launch of a persistent grid
//    that walks a tile list (system, site block) (hop_batch_kernel); the
//    vector steps are batched the same way;
//  * per-system arguments, solver state and reduction scratch live in
//    device memory, so a chunk of CHUNK regular iterations has no host
//    dependency: it is captured once into a CUDA graph and replayed;
//  * reset steps run (uncaptured) when any system asks for one: double-float
//    intermediate resets with a binary64 confirmation, as in oq_cgne_solve
//    (binary64 only when OQ_OPT_DF64_RESETS is 0).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "../../include/oq.h"
#include "ctx.h"
#include "oq_kernels.h"
#include "reduce.cuh"

namespace oq {

struct VecSys {
  long Vh;
  char* p;      // small-type direction
  char* r;      // small-type residual
  char* xs;     // small-type solution (binary32, or binary64 for F64 solves)
  char* xd;     // binary64 solution
  char* rd;     // residual r_d: binary64, or double-float after a double-float reset
  CgState* cg;
  RedArgs red;
};

enum VecOp { VOP_P = 0, VOP_ACCX = 1, VOP_RESTART = 2, VOP_RESTART_DF = 3 };

static const int VT = 256;  // sites per vector tile

template <int P, int XP, int OP>
__global__ void __launch_bounds__(VT) vec_batch_kernel(const VecSys* __restrict__ sys, const int2* __restrict__ tiles,
                                                      int ntiles) {
  typedef typename PrecTraits<P>::R R;
  typedef typename PrecTraits<XP>::R RX;
  __shared__ double smem[VT / 32];
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int2 tl = tiles[t];
    const VecSys& v = sys[tl.x];
    const long i = (long)tl.y * VT + threadIdx.x;
    const int gate = OP == VOP_P ? MODE_RUN : MODE_RESET;
    const bool live = i < v.Vh && v.cg->mode == gate;
    double acc = 0.0;
    if (live) {
      if constexpr (OP == VOP_P) {
        const R beta = (R)v.cg->beta;
        Spinor<R> pv, rv;
        load_spinor<P>(v.p, v.Vh, i, pv);
        load_spinor<P>(v.r, v.Vh, i, rv);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            pv.c[s][c].re = fma(beta, pv.c[s][c].re, rv.c[s][c].re);
            pv.c[s][c].im = fma(beta, pv.c[s][c].im, rv.c[s][c].im);
          }
        store_spinor<P>(v.p, v.Vh, i, pv);
      } else if constexpr (OP == VOP_ACCX) {
        const double sc = v.cg->scale;
        Spinor<double> d;
        Spinor<RX> w;
        load_spinor<P_F64>(v.xd, v.Vh, i, d);
        load_spinor<XP>(v.xs, v.Vh, i, w);
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            d.c[s][c].re = fma(sc, (double)w.c[s][c].re, d.c[s][c].re);
            d.c[s][c].im = fma(sc, (double)w.c[s][c].im, d.c[s][c].im);
          }
        store_spinor<P_F64>(v.xd, v.Vh, i, d);
      } else {
        const double inv = 1.0 / v.cg->scale;
        Spinor<R> q;
        Spinor<RX> z;
        if constexpr (OP == VOP_RESTART_DF) {
          Spinor<dfloat> d;
          load_spinor<P_DF64>(v.rd, v.Vh, i, d);
          const float invf = (float)inv;
#pragma unroll
          for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c)
              q.c[s][c] = cx<R>{(R)(__fadd_rn(d.c[s][c].re.hi, d.c[s][c].re.lo) * invf),
                                (R)(__fadd_rn(d.c[s][c].im.hi, d.c[s][c].im.lo) * invf)};
        } else {
          Spinor<double> d;
          load_spinor<P_F64>(v.rd, v.Vh, i, d);
#pragma unroll
          for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) q.c[s][c] = cx<R>{(R)(d.c[s][c].re * inv), (R)(d.c[s][c].im * inv)};
        }
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
          for (int c = 0; c < 3; ++c) z.c[s][c] = cx<RX>{0, 0};
        round_trip<P>(q);
        store_spinor<P>(v.r, v.Vh, i, q);
        store_spinor<P>(v.p, v.Vh, i, q);
        store_spinor<XP>(v.xs, v.Vh, i, z);
        acc = site_norm2(q);
      }
    }
    if constexpr (OP == VOP_RESTART || OP == VOP_RESTART_DF) {
      const unsigned nblk = (unsigned)((v.Vh + VT - 1) / VT);
      grid_reduce(acc, v.red, 0, 1, smem, (unsigned)tl.y, nblk);
    }
  }
}

template <int P, int XP>
static cudaError_t vec_batch(int op, const VecSys* sys, const int2* tiles, int ntiles, int grid, cudaStream_t s) {
  switch (op) {
    case VOP_P: vec_batch_kernel<P, XP, VOP_P><<<grid, VT, 0, s>>>(sys, tiles, ntiles); break;
    case VOP_ACCX: vec_batch_kernel<P, XP, VOP_ACCX><<<grid, VT, 0, s>>>(sys, tiles, ntiles); break;
    case VOP_RESTART: vec_batch_kernel<P, XP, VOP_RESTART><<<grid, VT, 0, s>>>(sys, tiles, ntiles); break;
    default:
      if constexpr (P == P_F64) return cudaErrorInvalidValue;  // binary64 solves reset in binary64
      else vec_batch_kernel<P, XP, VOP_RESTART_DF><<<grid, VT, 0, s>>>(sys, tiles, ntiles);
      break;
  }
  return cudaGetLastError();
}

static cudaError_t vec_batch_any(int prec, int op, const VecSys* sys, const int2* tiles, int ntiles, int grid,
                                 cudaStream_t s) {
  switch (prec) {
    case P_F64: return vec_batch<P_F64, P_F64>(op, sys, tiles, ntiles, grid, s);
    case P_F32: return vec_batch<P_F32, P_F32>(op, sys, tiles, ntiles, grid, s);
    case P_BF16: return vec_batch<P_BF16, P_F32>(op, sys, tiles, ntiles, grid, s);
    case P_F16: return vec_batch<P_F16, P_F32>(op, sys, tiles, ntiles, grid, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace oq

using namespace oq;

namespace {
const int BCHUNK = 8;
double batch_default_delta(int prec) {
  const double eps = prec == P_F32 ? ldexp(1.0, -23) : prec == P_BF16 ? ldexp(1.0, -7)
                   : prec == P_F16 ? ldexp(1.0, -10) : 0.0;
  const double d = 10.0 * eps;
  return d > 0.1 ? 0.1 : d;
}
}  // namespace

extern "C" int oq_cgne_solve_batch(oq_handle h, int nsys, const int* lats, const oq_solver_params* prm,
                                   const double* const* eta_dev, double* const* psi_dev, oq_status* st,
                                   void* stream) {
  if (!h || nsys < 1 || nsys > 64 || !lats || !prm || !eta_dev || !psi_dev || !st) return OQ_ERR_ARG;
  const int P = prm->sdtype;
  if (P < 0 || P > 3 || !(prm->res > 0.0) || prm->nmx < 1 || prm->nladder != 0) return OQ_ERR_ARG;
  int fmt = -1;
  for (int s = 0; s < nsys; ++s) {
    if (lats[s] < 0 || lats[s] >= (int)h->lats.size() || !eta_dev[s] || !psi_dev[s]) return OQ_ERR_ARG;
    const LatCtx& L = h->lats[lats[s]];
    if (!L.has_clover || L.halo_t) return OQ_ERR_STATE;  // whole lattices only
    if (fmt < 0) fmt = L.link_fmt;
    if (L.link_fmt != fmt) return OQ_ERR_ARG;  // one link format per batch (one kernel instantiation)
  }
  cudaStream_t us = (cudaStream_t)stream;
  if (cudaStreamSynchronize(us) != cudaSuccess) return OQ_ERR_CUDA;
  int rc = h->ensure_work_stream();
  if (rc) return rc;
  cudaStream_t s = h->work_stream;
  const int XP = P == P_F64 ? P_F64 : P_F32;
  const int bx_lo = 128, bx_64 = 64;
  // per-system buffers
  std::vector<long> Vh(nsys);
  std::vector<void*> eta64(nsys), xd(nsys), rd(nsys), t64(nsys), u64v(nsys), pv(nsys), rv(nsys), uv(nsys),
      tv(nsys), xs(nsys), xdf(nsys), etadf(nsys);
  // double-float intermediate resets (binary64 confirmation), as oq_cgne_solve
  int reset_prec = (P != P_F64 && h->df64_resets) ? P_DF64 : P_F64;
  if (reset_prec == P_DF64)
    for (int s2 = 0; s2 < nsys; ++s2) {
      rc = h->ensure_df(lats[s2], s);
      if (rc) return rc;
    }
  long maxblk = 1;
  for (int s2 = 0; s2 < nsys; ++s2) {
    const int lat = lats[s2];
    Vh[s2] = h->lats[lat].g.Vh;
    const size_t h64 = spinor_half_bytes(Vh[s2], P_F64), hP = spinor_half_bytes(Vh[s2], P),
                 hX = spinor_half_bytes(Vh[s2], XP);
    const std::string k = "bcg" + std::to_string(s2) + "_";
    rc |= h->workspace(lat, (k + "eta64").c_str(), h64, &eta64[s2]);
    rc |= h->workspace(lat, (k + "xd").c_str(), h64, &xd[s2]);
    rc |= h->workspace(lat, (k + "rd").c_str(), h64, &rd[s2]);
    rc |= h->workspace(lat, (k + "t64").c_str(), h64, &t64[s2]);
    rc |= h->workspace(lat, (k + "u64").c_str(), h64, &u64v[s2]);
    rc |= h->workspace(lat, (k + "p").c_str(), hP, &pv[s2]);
    rc |= h->workspace(lat, (k + "r").c_str(), hP, &rv[s2]);
    rc |= h->workspace(lat, (k + "u").c_str(), hP, &uv[s2]);
    rc |= h->workspace(lat, (k + "t").c_str(), hP, &tv[s2]);
    rc |= h->workspace(lat, (k + "xs").c_str(), hX, &xs[s2]);
    if (reset_prec == P_DF64) {
      rc |= h->workspace(lat, (k + "xdf").c_str(), h64, &xdf[s2]);
      rc |= h->workspace(lat, (k + "etadf").c_str(), h64, &etadf[s2]);
    }
    const long nb = (Vh[s2] + 31) / 32;
    if (nb > maxblk) maxblk = nb;
  }
  if (rc) return OQ_ERR_NOMEM;
  // batch scratch (on lattice 0's workspace): partials, counters, results, states, args, tiles
  void *bpart, *bcnt, *bres, *bcg, *bargs, *bvsys, *btiles;
  const int NARG = 12;
  std::vector<int2> tiles_lo, tiles_64, tiles_v;
  for (int s2 = 0; s2 < nsys; ++s2) {
    for (long b = 0; b < (Vh[s2] + bx_lo - 1) / bx_lo; ++b) tiles_lo.push_back(make_int2(s2, (int)b));
    for (long b = 0; b < (Vh[s2] + bx_64 - 1) / bx_64; ++b) tiles_64.push_back(make_int2(s2, (int)b));
    for (long b = 0; b < (Vh[s2] + 255) / 256; ++b) tiles_v.push_back(make_int2(s2, (int)b));
  }
  rc |= h->workspace(lats[0], "b_part", sizeof(double) * nsys * maxblk, &bpart);
  rc |= h->workspace(lats[0], "b_cnt", sizeof(unsigned) * nsys, &bcnt);
  rc |= h->workspace(lats[0], "b_res", sizeof(double) * nsys, &bres);
  rc |= h->workspace(lats[0], "b_cg", sizeof(CgState) * nsys, &bcg);
  rc |= h->workspace(lats[0], "b_args", sizeof(HopArgs) * NARG * nsys, &bargs);
  rc |= h->workspace(lats[0], "b_vsys", sizeof(VecSys) * 4 * nsys, &bvsys);
  rc |= h->workspace(lats[0], "b_tiles", sizeof(int2) * (tiles_lo.size() + tiles_64.size() + tiles_v.size()),
                     &btiles);
  if (rc) return OQ_ERR_NOMEM;
  int2* t_lo = (int2*)btiles;
  int2* t_64 = t_lo + tiles_lo.size();
  int2* t_v = t_64 + tiles_64.size();

#define CK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) return OQ_ERR_CUDA; \
  } while (0)
#define KL(x)                                   \
  do {                                          \
    h->launches += 1;                           \
    if ((x) != cudaSuccess) return OQ_ERR_CUDA; \
  } while (0)

  CK(cudaMemsetAsync(bcnt, 0, sizeof(unsigned) * nsys, s));
  CK(cudaMemcpyAsync(t_lo, tiles_lo.data(), sizeof(int2) * tiles_lo.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(t_64, tiles_64.data(), sizeof(int2) * tiles_64.size(), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(t_v, tiles_v.data(), sizeof(int2) * tiles_v.size(), cudaMemcpyHostToDevice, s));

  CgState* cg = (CgState*)bcg;
  auto red_for = [&](int s2, int fin, int gate) {
    RedArgs r;
    r.partials = (double*)bpart + (long)s2 * maxblk;
    r.counters = (unsigned*)bcnt + s2;
    r.result = (double*)bres + s2;
    r.cg = cg + s2;
    r.fin = fin;
    r.gate = gate;
    return r;
  };
  // argument sets: 0 P1, 1 P2+norm, 2 P1^dag, 3 P2^dag+CG (small type); 4..7 the binary64 reset
  // passes; 8..11 the double-float reset passes (split x_d and eta in, r_d out as double-float)
  std::vector<HopArgs> args((size_t)NARG * nsys);
  for (int s2 = 0; s2 < nsys; ++s2) {
    const int lat = lats[s2];
    const long hP = spinor_half_bytes(Vh[s2], P), h64 = spinor_half_bytes(Vh[s2], P_F64),
               hX = spinor_half_bytes(Vh[s2], XP);
    HopArgs base = h->hop_args(lat, P);
    base.cg = cg + s2;
    base.gate = MODE_RUN;
    base.half_bytes = hP;
    HopArgs a = base;
    a.in = pv[s2]; a.out = tv[s2]; a.p = 1;
    args[0 * nsys + s2] = a;
    a = base;
    a.in = tv[s2]; a.in2 = pv[s2]; a.out = uv[s2]; a.p = 0;
    a.red = red_for(s2, FIN_ALPHA, MODE_RUN);
    args[1 * nsys + s2] = a;
    a = base;
    a.in = uv[s2]; a.out = tv[s2]; a.p = 1;
    args[2 * nsys + s2] = a;
    a = base;
    a.in = tv[s2]; a.in2 = uv[s2]; a.p = 0;
    a.ep_x = xs[s2]; a.ep_p = pv[s2]; a.ep_r = rv[s2];
    a.red = red_for(s2, FIN_BETA, MODE_RUN);
    args[3 * nsys + s2] = a;
    HopArgs b64 = h->hop_args(lat, P_F64);
    b64.cg = cg + s2;
    b64.gate = MODE_RESET;
    b64.half_bytes = h64;
    a = b64;
    a.in = xd[s2]; a.out = t64[s2]; a.p = 1;
    args[4 * nsys + s2] = a;
    a = b64;
    a.in = t64[s2]; a.in2 = xd[s2]; a.out = u64v[s2]; a.p = 0;
    args[5 * nsys + s2] = a;
    a = b64;
    a.in = u64v[s2]; a.out = t64[s2]; a.p = 1;
    args[6 * nsys + s2] = a;
    a = b64;
    a.in = t64[s2]; a.in2 = u64v[s2]; a.out = rd[s2]; a.p = 0;
    a.ep_eta = eta64[s2];
    a.red = red_for(s2, FIN_RD2, MODE_RESET);
    args[7 * nsys + s2] = a;
    if (reset_prec == P_DF64) {
      HopArgs bdf = h->hop_args(lat, P_DF64);
      bdf.cg = cg + s2;
      bdf.gate = MODE_RESET;
      bdf.half_bytes = h64;
      a = bdf;
      a.in = xdf[s2]; a.out = t64[s2]; a.p = 1;
      args[8 * nsys + s2] = a;
      a = bdf;
      a.in = t64[s2]; a.in2 = xdf[s2]; a.out = u64v[s2]; a.p = 0;
      args[9 * nsys + s2] = a;
      a = bdf;
      a.in = u64v[s2]; a.out = t64[s2]; a.p = 1;
      args[10 * nsys + s2] = a;
      a = bdf;
      a.in = t64[s2]; a.in2 = u64v[s2]; a.out = rd[s2]; a.p = 0;
      a.ep_eta = etadf[s2];
      a.red = red_for(s2, FIN_RD2, MODE_RESET);
      args[11 * nsys + s2] = a;
    }
    (void)hX;
  }
  CK(cudaMemcpyAsync(bargs, args.data(), sizeof(HopArgs) * args.size(), cudaMemcpyHostToDevice, s));
  std::vector<VecSys> vs((size_t)4 * nsys);
  for (int s2 = 0; s2 < nsys; ++s2) {
    VecSys v;
    v.Vh = Vh[s2];
    v.p = (char*)pv[s2];
    v.r = (char*)rv[s2];
    v.xs = (char*)xs[s2];
    v.xd = (char*)xd[s2];
    v.rd = (char*)rd[s2];
    v.cg = cg + s2;
    v.red = red_for(s2, FIN_STORE, 0);
    vs[0 * nsys + s2] = v;  // VOP_P
    vs[1 * nsys + s2] = v;  // VOP_ACCX
    v.red = red_for(s2, FIN_RESTART, MODE_RESET);
    vs[2 * nsys + s2] = v;  // VOP_RESTART
    vs[3 * nsys + s2] = v;  // VOP_RESTART_DF
  }
  CK(cudaMemcpyAsync(bvsys, vs.data(), sizeof(VecSys) * vs.size(), cudaMemcpyHostToDevice, s));
  const HopArgs* dargs = (const HopArgs*)bargs;
  const VecSys* dvs = (const VecSys*)bvsys;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  const int grid_lo = (int)std::min<long>((long)tiles_lo.size(), (long)nsm * 8);
  const int grid_64 = (int)std::min<long>((long)tiles_64.size(), (long)nsm * 8);
  const int grid_v = (int)std::min<long>((long)tiles_v.size(), (long)nsm * 8);

  auto hop = [&](int argset, int prec, int mode, int dag, int epi) -> cudaError_t {
    HopLaunch l;
    l.prec = prec;
    l.link_fmt = fmt;
    l.mode = mode;
    l.dagger = dag;
    l.epi = epi;
    const bool f64 = prec == P_F64 || prec == P_DF64;
    l.bx = f64 ? bx_64 : bx_lo;
    l.by = 1;
    l.sys = dargs + (long)argset * nsys;
    l.tiles = f64 ? t_64 : t_lo;
    l.ntiles = (int)(f64 ? tiles_64.size() : tiles_lo.size());
    l.grid = f64 ? grid_64 : grid_lo;
    HopArgs dummy;
    memset(&dummy, 0, sizeof(dummy));
    h->launches += 1;
    return launch_hop(l, dummy, s);
  };

  // eta -> packed binary64, initial state
  std::vector<double> eta_n(nsys);
  {
    RedArgs ra = h->red_args(FIN_STORE, 0);
    rc = h->ensure_reduce(2, reduce_grid(maxblk * 32));
    if (rc) return rc;
    for (int s2 = 0; s2 < nsys; ++s2) {
      const LatCtx& L = h->lats[lats[s2]];
      const long h64 = spinor_half_bytes(Vh[s2], P_F64);
      KL(pack_spinor(L.g, P_F64, OQ_EVEN, eta_dev[s2], eta64[s2], 1.0, 1, 2 * Vh[s2] * 12, h64, s));
      CK(cudaMemsetAsync(xd[s2], 0, h64, s));
      CK(cudaMemsetAsync(xs[s2], 0, spinor_half_bytes(Vh[s2], XP), s));
      CK(cudaMemcpyAsync(rd[s2], eta64[s2], h64, cudaMemcpyDeviceToDevice, s));
      if (reset_prec == P_DF64) KL(split_f64((const double*)eta64[s2], etadf[s2], h64 / sizeof(double), s));
      ra = h->red_args(FIN_STORE, 0);
      KL(reduce_norm2(P_F64, eta64[s2], Vh[s2], h64, 1, ra, s));
      double v = 0.0;
      CK(cudaMemcpyAsync(h->results_host, h->results, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      v = h->results_host[0];
      eta_n[s2] = sqrt(v);
    }
  }
  rc = h->ensure_cg(nsys);
  if (rc) return rc;
  CgState* cs = h->cg_host;
  const double delta = prm->delta > 0.0 ? prm->delta : batch_default_delta(P);
  std::vector<int> resets(nsys, 0);
  for (int s2 = 0; s2 < nsys; ++s2) {
    memset(&cs[s2], 0, sizeof(CgState));
    cs[s2].mode = MODE_RESET;
    cs[s2].rd2 = eta_n[s2] * eta_n[s2];
    cs[s2].nmx = prm->nmx;
    cs[s2].delta2 = delta * delta;
  }
  auto decide = [&](bool count) -> int {
    int pending = 0;
    for (int k = 0; k < nsys; ++k) {
      CgState& c = cs[k];
      if (c.mode != MODE_RESET) continue;
      if (count) resets[k] += 1;
      const double rn = sqrt(c.rd2);
      if (!isfinite(c.rd2) || eta_n[k] == 0.0 || rn <= prm->res * eta_n[k] || c.steps >= prm->nmx ||
          resets[k] > prm->nmx) {
        c.mode = MODE_DONE;
        continue;
      }
      c.scale = rn / sqrt(12.0 * (double)Vh[k]);
      const double t = prm->res * eta_n[k] / c.scale;
      c.tol2 = t * t;
      ++pending;
    }
    return pending;
  };
  auto upload = [&]() -> int {
    CK(cudaMemcpyAsync(cg, cs, sizeof(CgState) * nsys, cudaMemcpyHostToDevice, s));
    return OQ_OK;
  };
  auto download = [&]() -> int {
    CK(cudaMemcpyAsync(cs, cg, sizeof(CgState) * nsys, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return OQ_OK;
  };
  // storage of r_d (every system that restarts was reset by the latest reset step)
  int rd_prec = P_F64;
  auto restart = [&]() -> int {
    if (rd_prec == P_DF64)
      KL(vec_batch_any(P, VOP_RESTART_DF, dvs + 3 * nsys, t_v, (int)tiles_v.size(), grid_v, s));
    else
      KL(vec_batch_any(P, VOP_RESTART, dvs + 2 * nsys, t_v, (int)tiles_v.size(), grid_v, s));
    return OQ_OK;
  };
  // rp: arithmetic of the residual recomputation; accumulate: add s x_s to
  // x_d first (false re-checks the same x_d in binary64)
  auto reset_step = [&](int rp, bool accumulate) -> int {
    if (accumulate) KL(vec_batch_any(P, VOP_ACCX, dvs + 1 * nsys, t_v, (int)tiles_v.size(), grid_v, s));
    if (rp == P_DF64) {
      for (int s2 = 0; s2 < nsys; ++s2)
        KL(split_f64((const double*)xd[s2], xdf[s2], spinor_half_bytes(Vh[s2], P_F64) / sizeof(double), s));
      CK(hop(8, P_DF64, HOP_P1, 0, EPI_NONE));
      CK(hop(9, P_DF64, HOP_P2, 0, EPI_NONE));
      CK(hop(10, P_DF64, HOP_P1, 1, EPI_NONE));
      CK(hop(11, P_DF64, HOP_P2, 1, EPI_RESID64));
    } else {
      CK(hop(4, P_F64, HOP_P1, 0, EPI_NONE));
      CK(hop(5, P_F64, HOP_P2, 0, EPI_NONE));
      CK(hop(6, P_F64, HOP_P1, 1, EPI_NONE));
      CK(hop(7, P_F64, HOP_P2, 1, EPI_RESID64));
    }
    rd_prec = rp;
    return OQ_OK;
  };
  auto iteration = [&]() -> cudaError_t {
    cudaError_t e;
    if ((e = hop(0, P, HOP_P1, 0, EPI_NONE)) != cudaSuccess) return e;
    if ((e = hop(1, P, HOP_P2, 0, EPI_NORM)) != cudaSuccess) return e;
    if ((e = hop(2, P, HOP_P1, 1, EPI_NONE)) != cudaSuccess) return e;
    if ((e = hop(3, P, HOP_P2, 1, EPI_CG)) != cudaSuccess) return e;
    h->launches += 1;
    return vec_batch_any(P, VOP_P, dvs, t_v, (int)tiles_v.size(), grid_v, s);
  };

  // capture CHUNK regular iterations once
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  {
    const long long l0 = h->launches;
    CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    cudaError_t ce = cudaSuccess;
    for (int k = 0; k < BCHUNK && ce == cudaSuccess; ++k) ce = iteration();
    cudaError_t ee = cudaStreamEndCapture(s, &graph);
    if (ce != cudaSuccess || ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return OQ_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&gexec, graph, 0) != cudaSuccess) {
      cudaGraphDestroy(graph);
      return OQ_ERR_CUDA;
    }
    h->launches = l0;  // captured, not launched
  }
  const long long per_chunk = (long long)BCHUNK * 5;
  int ret = OQ_OK;
  auto body = [&]() -> int {
    int pending = decide(false);
    int r2 = upload();
    if (r2) return r2;
    if (pending) {
      r2 = restart();
      if (r2) return r2;
    }
    for (;;) {
      r2 = download();
      if (r2) return r2;
      int run = 0, rst = 0;
      for (int k = 0; k < nsys; ++k) {
        run += cs[k].mode == MODE_RUN;
        rst += cs[k].mode == MODE_RESET;
      }
      if (rst) {
        // a reset whose inner solves all stopped on the target is expected to
        // end the solve: binary64 right away, not double-float plus confirmation
        int rp = reset_prec;
        if (rp == P_DF64) {
          bool all_tol = true;
          for (int k = 0; k < nsys; ++k)
            if (cs[k].mode == MODE_RESET && cs[k].reason != WHY_TOL) all_tol = false;
          if (all_tol) rp = P_F64;
        }
        r2 = reset_step(rp, true);
        if (r2) return r2;
        r2 = download();
        if (r2) return r2;
        if (rp == P_DF64) {
          // a double-float residual may only propose convergence: confirm in binary64
          bool claims = false;
          for (int k = 0; k < nsys; ++k)
            if (cs[k].mode == MODE_RESET && sqrt(cs[k].rd2) <= prm->res * eta_n[k]) claims = true;
          if (claims) {
            std::vector<double> df(nsys);
            for (int k = 0; k < nsys; ++k) df[k] = cs[k].rd2;
            r2 = reset_step(P_F64, false);
            if (r2) return r2;
            r2 = download();
            if (r2) return r2;
            for (int k = 0; k < nsys; ++k)
              if (cs[k].mode == MODE_RESET && sqrt(df[k]) <= prm->res * eta_n[k] &&
                  sqrt(cs[k].rd2) > prm->res * eta_n[k])
                reset_prec = P_F64;
          }
        }
        pending = decide(true);
        r2 = upload();
        if (r2) return r2;
        if (pending) {
          r2 = restart();
          if (r2) return r2;
        }
        continue;
      }
      if (!run) break;
      if (cudaGraphLaunch(gexec, s) != cudaSuccess) return OQ_ERR_CUDA;
      h->launches += per_chunk;
    }
    return OQ_OK;
  };
  ret = body();
  cudaGraphExecDestroy(gexec);
  cudaGraphDestroy(graph);
  if (ret) return ret;
  for (int s2 = 0; s2 < nsys; ++s2) {
    const LatCtx& L = h->lats[lats[s2]];
    CK(cudaMemsetAsync(psi_dev[s2], 0, sizeof(double) * 24 * 2 * Vh[s2], s));
    KL(unpack_spinor(L.g, P_F64, OQ_EVEN, xd[s2], psi_dev[s2], 1.0, 1, spinor_half_bytes(Vh[s2], P_F64),
                     2 * Vh[s2] * 12, s));
  }
  CK(cudaStreamSynchronize(s));
  for (int k = 0; k < nsys; ++k) {
    st[k].steps = cs[k].steps;
    st[k].resets = resets[k];
    st[k].restarts = 0;
    st[k].cycles = 0;
    st[k].mr_avg = 0.0;
    st[k].nn_fallback = 0;
    for (int i = 0; i < 4; ++i) st[k].ladder_steps[i] = i == 0 ? cs[k].steps : 0;
    st[k].true_rel_res = eta_n[k] > 0.0 ? sqrt(cs[k].rd2) / eta_n[k] : 0.0;
    st[k].converged = (isfinite(cs[k].rd2) && st[k].true_rel_res <= prm->res) ? 1 : 0;
    if (!isfinite(cs[k].rd2)) ret = OQ_ERR_NONFINITE;
    else if (!st[k].converged && ret == OQ_OK) ret = OQ_ERR_NOCONV;
  }
  return ret;
#undef CK
#undef KL
}
