// CGNE with reset steps (Sec. 2 and the caption of Fig. 4).
//
// Solves A psi = eta, A = Dhat^dag Dhat, on the even sites.  Regular CG steps
// run with vectors stored in the small type (binary32, bfloat16 or binary16;
// binary32 arithmetic), every reduction is binary64.  The small-type CG
// solves A x_s = r_d / s for the current binary64 residual r_d, scaled by
// s = ||r_d|| / sqrt(12 Ve) so that stored components are O(1).  A reset step
// adds s x_s to the binary64 solution x_d and recomputes r_d = eta - A x_d
// once the recursive residual has dropped below delta times its value at the
// previous reset (delta ~ 10 eps of the small type), reached the target, or
// nmx steps are used.  The paper recomputes r_d in binary64; here the
// intermediate recomputations use double-float arithmetic (~48 bits, on the
// binary32 pipes, 3x faster than binary64 on GB300) unless
// OQ_OPT_DF64_RESETS is 0, and a residual that meets the target is always
// confirmed by a binary64 recomputation (a reset whose inner solves stopped
// on the target is computed in binary64 right away).  The regular steps never
// wait for the host: alpha, beta and the reset decision are computed on the
// device by the last CTA of each fused grid reduction; the host looks at the
// per-rhs state after a chunk of iterations.  The chunk is the number of
// steps left until the earliest predicted end of an inner solve (its length
// predicted as one less than the previous inner solve of that rhs; at most
// CHUNK, at least 1): an iteration launched after every rhs has stopped is
// gated off on the device and does nothing, but still costs the launch of
// every CTA, while a look at the state costs one small copy.
//
// Precision ladder (Sec. 2, after Fig. 4): the storage type of the regular
// steps may change from one inner solve to the next, e.g. binary16 until the
// binary64 residual is below eps(binary16) ||eta||, then binary32, then
// binary64.  All right-hand sides of one call share the kernels of one type
// (the phase): a right-hand side whose reset qualifies it for the next type
// is parked (no kernel acts on it) until every other one is parked or done;
// then the phase advances and the parked ones restart in the new type.  Each
// right-hand side thus runs the same sequence of inner solves as alone.
//
// One iteration = 5 launches:
//   P1(p -> t)  ;  P2(t, p -> u = Dhat p) + ||u||^2 -> alpha
//   P1^dag(u -> t) ; P2^dag(t, u -> q) fused with x += alpha p, r -= alpha q,
//   ||r||^2 -> beta / stop test  ;  p = r + beta p
#include <math.h>
#include <string.h>

#include <vector>

#include "../../include/oq.h"
#include "ctx.h"
#include "oq_kernels.h"

using namespace oq;

namespace {

const int CHUNK = 8;   // chunk length before a rhs has a previous inner solve, and the maximum

// unit of least precision at 1 of a storage type (0 for binary64 storage)
double type_eps(int prec) {
  return prec == P_F32 ? ldexp(1.0, -23) : prec == P_BF16 ? ldexp(1.0, -7)
       : prec == P_F16 ? ldexp(1.0, -10) : 0.0;
}

double default_delta(int prec) {
  double d = 10.0 * type_eps(prec);
  return d > 0.1 ? 0.1 : d;
}

}  // namespace

// eta / psi of the solvers: device memory, or page-locked host memory that
// CUDA maps into the device's address space at the same address (the pack
// and unpack kernels then read and write it over the host link themselves)
static bool kernel_addressable(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return true;
  return at.type == cudaMemoryTypeHost && at.devicePointer == p;
}

// half: eta / psi hold the even sites only (lexicographic index / 2)
static int cgne_impl(oq_handle h, int lat, const oq_solver_params* prm, const double* eta_dev, double* psi_dev,
                     int nrhs, oq_status* st, void* stream, int half) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || !prm || !eta_dev || !psi_dev || nrhs < 1 || !st) return OQ_ERR_ARG;
  if (!(prm->res > 0.0) || prm->nmx < 1 || prm->nladder < 0 || prm->nladder > 4) return OQ_ERR_ARG;
  if (!kernel_addressable(eta_dev) || !kernel_addressable(psi_dev)) return OQ_ERR_ARG;
  // the storage types of the phases: sdtype alone, or the ladder
  std::vector<int> phase_prec;
  if (prm->nladder == 0) phase_prec.push_back(prm->sdtype);
  for (int i = 0; i < prm->nladder; ++i) phase_prec.push_back(prm->ladder[i]);
  for (int q : phase_prec)
    if (q < 0 || q > 3) return OQ_ERR_ARG;
  const double ladder_c = prm->ladder_c > 0.0 ? prm->ladder_c : 1.0;
  const int nphase = (int)phase_prec.size();
  int phase = 0;
  LatCtx& L = h->lats[lat];
  if (!L.has_clover || L.halo_t) return OQ_ERR_STATE;  // whole lattices only
  cudaStream_t s = (cudaStream_t)stream;
  const long Vh = L.g.Vh;
  // small type of the current phase (P), its solution type (XP) and sizes;
  // buffers are sized for the largest type of any phase
  int P = phase_prec[0];
  int XP = P == P_F64 ? P_F64 : P_F32;
  const size_t h64 = spinor_half_bytes(Vh, P_F64);
  size_t hP = spinor_half_bytes(Vh, P), hX = spinor_half_bytes(Vh, XP);
  size_t hPmax = 0, hXmax = 0;
  for (int q : phase_prec) {
    const size_t a = spinor_half_bytes(Vh, q), b = spinor_half_bytes(Vh, q == P_F64 ? P_F64 : P_F32);
    hPmax = a > hPmax ? a : hPmax;
    hXmax = b > hXmax ? b : hXmax;
  }
  const size_t canon_field = sizeof(double) * 24 * (half ? 1 : 2) * Vh;
  const long canon_stride = (half ? 1 : 2) * Vh * 12;  // double2 per canonical field
  void *eta64, *xd, *rd, *t64, *u64v, *pv, *rv, *uv, *tv, *xs;
  int rc = 0;
  rc |= h->workspace(lat, "cg_eta64", h64 * nrhs, &eta64);
  rc |= h->workspace(lat, "cg_xd", h64 * nrhs, &xd);
  rc |= h->workspace(lat, "cg_rd", h64 * nrhs, &rd);
  rc |= h->workspace(lat, "cg_t64", h64 * nrhs, &t64);
  rc |= h->workspace(lat, "cg_u64", h64 * nrhs, &u64v);
  rc |= h->workspace(lat, "cg_p", hPmax * nrhs, &pv);
  rc |= h->workspace(lat, "cg_r", hPmax * nrhs, &rv);
  rc |= h->workspace(lat, "cg_u", hPmax * nrhs, &uv);
  rc |= h->workspace(lat, "cg_t", hPmax * nrhs, &tv);
  rc |= h->workspace(lat, "cg_xs", hXmax * nrhs, &xs);
  if (rc) return OQ_ERR_NOMEM;
  const long grid_hop = (Vh + 31) / 32;  // upper bound on CTAs of any stencil launch
  rc = h->ensure_reduce(2 * nrhs, grid_hop > reduce_grid(Vh) ? grid_hop : reduce_grid(Vh));
  if (!rc) rc = h->ensure_cg(nrhs);
  if (rc) return rc;

#define CK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) return OQ_ERR_CUDA; \
  } while (0)
#define KL(x)                                   \
  do {                                          \
    h->launches += 1;                           \
    if ((x) != cudaSuccess) return OQ_ERR_CUDA; \
  } while (0)
#define RK(x)              \
  do {                     \
    int rc_ = (x);         \
    if (rc_) return rc_;   \
  } while (0)

  // eta -> packed binary64 even field; x_d = 0, x_s = 0
  KL(pack_spinor(L.g, P_F64, OQ_EVEN, eta_dev, eta64, 1.0, nrhs, canon_stride, (long)h64, s, half));
  CK(cudaMemsetAsync(xd, 0, h64 * nrhs, s));
  CK(cudaMemsetAsync(xs, 0, hXmax * nrhs, s));
  CK(cudaMemcpyAsync(rd, eta64, h64 * nrhs, cudaMemcpyDeviceToDevice, s));
  {
    RedArgs ra = h->red_args(FIN_STORE, 0);
    KL(reduce_norm2(P_F64, eta64, Vh, (long)h64, nrhs, ra, s));
  }
  CK(cudaMemcpyAsync(h->results_host, h->results, sizeof(double) * nrhs, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::vector<double> eta_n(nrhs);
  std::vector<int> resets(nrhs, 0);
  std::vector<int> phase_steps(4 * (size_t)nrhs, 0), steps_before(nrhs, 0);
  const double ncomp = 12.0 * (double)Vh;
  CgState* cs = h->cg_host;
  for (int k = 0; k < nrhs; ++k) {
    eta_n[k] = sqrt(h->results_host[k]);
    memset(&cs[k], 0, sizeof(CgState));
    cs[k].mode = MODE_RESET;
    cs[k].rd2 = h->results_host[k];
    cs[k].nmx = prm->nmx;
  }
  // diagnostics (OQ_OPT_HISTORY): the recursive residual of every regular step
  // (recorded on the device by the p update) and the residual of every reset
  double* hist = nullptr;
  const int hcap = prm->nmx < 100000 ? prm->nmx : 100000;
  std::vector<std::vector<double>> reset_hist;
  if (h->history) {
    RK(h->workspace(lat, "cg_hist", sizeof(double) * (size_t)hcap * nrhs, (void**)&hist));
    CK(cudaMemsetAsync(hist, 0, sizeof(double) * (size_t)hcap * nrhs, s));
    reset_hist.assign(nrhs, {});
  }

  // decide, per rhs in MODE_RESET, between DONE, PARK (a later phase of the
  // ladder) and a restart of the small CG in the current phase
  auto decide = [&](bool count) -> int {
    int pending = 0;
    const double delta = prm->delta > 0.0 ? prm->delta : default_delta(P);
    const double sw = phase + 1 < nphase ? ladder_c * type_eps(P) : 0.0;
    for (int k = 0; k < nrhs; ++k) {
      CgState& c = cs[k];
      if (c.mode != MODE_RESET) continue;
      if (count) resets[k] += 1;
      const double rn = sqrt(c.rd2);
      if (!isfinite(c.rd2) || eta_n[k] == 0.0 || rn <= prm->res * eta_n[k] || c.steps >= prm->nmx ||
          resets[k] > prm->nmx) {
        c.mode = MODE_DONE;
        continue;
      }
      if (rn <= sw * eta_n[k]) {
        c.mode = MODE_PARK;
        continue;
      }
      c.delta2 = delta * delta;
      c.scale = rn / sqrt(ncomp);
      const double t = prm->res * eta_n[k] / c.scale;
      c.tol2 = t * t;
      ++pending;
    }
    return pending;
  };

  auto upload = [&]() -> int {
    CK(cudaMemcpyAsync(h->cg_dev, cs, sizeof(CgState) * nrhs, cudaMemcpyHostToDevice, s));
    return OQ_OK;
  };
  auto download = [&]() -> int {
    CK(cudaMemcpyAsync(cs, h->cg_dev, sizeof(CgState) * nrhs, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return OQ_OK;
  };
  // storage of r_d per rhs: binary64, or double-float after a double-float
  // reset.  The rhs that restart together share it: they were reset by the
  // same reset step, or (parked rhs at a phase change) are made to share it.
  std::vector<int> rd_fmt(nrhs, P_F64);
  auto restart = [&]() -> int {
    int rd_prec = -1;
    for (int k = 0; k < nrhs; ++k)
      if (cs[k].mode == MODE_RESET) {
        if (rd_prec >= 0 && rd_fmt[k] != rd_prec) return OQ_ERR_STATE;
        rd_prec = rd_fmt[k];
      }
    if (rd_prec < 0) return OQ_OK;
    RedArgs ra = h->red_args(FIN_RESTART, MODE_RESET);
    KL(cg_restart(P, rd, rd_prec, rv, pv, xs, XP, Vh, (long)h64, (long)hP, (long)hX, nrhs, ra, s));
    return OQ_OK;
  };

  // the reset step for all rhs in MODE_RESET.  rp: arithmetic of the residual
  // recomputation (binary64 storage either way); accumulate: add s x_s to x_d
  // first (false re-checks the same x_d)
  // double-float resets read the splits of x_d and eta and write r_d as
  // double-float (DF64 storage has the size of binary64)
  void *xdf = nullptr, *etadf = nullptr;
  auto reset_step = [&](int rp, bool accumulate) -> int {
    const void* xin = xd;
    const void* eta_in = eta64;
    if (rp == P_DF64) {
      RK(h->ensure_df(lat, s));
      if (!xdf) {
        RK(h->workspace(lat, "cg_xdf", h64 * nrhs, &xdf));
        RK(h->workspace(lat, "cg_etadf", h64 * nrhs, &etadf));
        KL(split_f64((const double*)eta64, etadf, h64 * nrhs / sizeof(double), s));
      }
      // the accumulation writes the split of x_d as well (for the rhs being reset)
      if (accumulate)
        KL(cg_accumulate_x(XP, (double*)xd, xs, Vh, (long)h64, (long)hX, nrhs, h->cg_dev, s, xdf));
      else
        KL(split_f64((const double*)xd, xdf, h64 * nrhs / sizeof(double), s));
      xin = xdf;
      eta_in = etadf;
    } else if (accumulate) {
      KL(cg_accumulate_x(XP, (double*)xd, xs, Vh, (long)h64, (long)hX, nrhs, h->cg_dev, s));
    }
    HopArgs a = h->hop_args(lat, rp);
    a.nrhs = nrhs;
    a.cg = h->cg_dev;
    a.gate = MODE_RESET;
    a.in_stride = a.in2_stride = a.out_stride = (long)h64;
    a.half_bytes = (long)h64;
    // t = A_oo^-1 D_oe x_d ; u = Dhat x_d
    a.in = xin; a.out = t64; a.p = 1;
    RK(h->run_hop(h->hop_launch(lat, rp, HOP_P1, 0, EPI_NONE, nrhs), a, s));
    a.in = t64; a.in2 = xin; a.out = u64v; a.p = 0;
    RK(h->run_hop(h->hop_launch(lat, rp, HOP_P2, 0, EPI_NONE, nrhs), a, s));
    // t = ..., r_d = eta - Dhat^dag u, ||r_d||^2
    a.in = u64v; a.out = t64; a.p = 1;
    RK(h->run_hop(h->hop_launch(lat, rp, HOP_P1, 1, EPI_NONE, nrhs), a, s));
    a.in = t64; a.in2 = u64v; a.out = rd; a.p = 0;
    a.ep_eta = eta_in; a.ep_eta_stride = (long)h64;
    a.red = h->red_args(FIN_RD2, MODE_RESET);
    RK(h->run_hop(h->hop_launch(lat, rp, HOP_P2, 1, EPI_RESID64, nrhs), a, s));
    for (int k = 0; k < nrhs; ++k)
      if (cs[k].mode == MODE_RESET) rd_fmt[k] = rp;
    return OQ_OK;
  };

  // one regular step for all rhs in MODE_RUN
  HopArgs it;
  auto set_phase_args = [&]() {
    it = h->hop_args(lat, P);
    it.nrhs = nrhs;
    it.cg = h->cg_dev;
    it.gate = MODE_RUN;
    it.in_stride = it.in2_stride = it.out_stride = (long)hP;
    it.half_bytes = (long)hP;
  };
  set_phase_args();
  auto iteration = [&]() -> int {
    HopArgs a = it;
    a.in = pv; a.out = tv; a.p = 1;
    RK(h->run_hop(h->hop_launch(lat, P, HOP_P1, 0, EPI_NONE, nrhs), a, s));
    a.in = tv; a.in2 = pv; a.out = uv; a.p = 0;
    a.red = h->red_args(FIN_ALPHA, MODE_RUN);
    RK(h->run_hop(h->hop_launch(lat, P, HOP_P2, 0, EPI_NORM, nrhs), a, s));
    a = it;
    a.in = uv; a.out = tv; a.p = 1;
    RK(h->run_hop(h->hop_launch(lat, P, HOP_P1, 1, EPI_NONE, nrhs), a, s));
    a.in = tv; a.in2 = uv; a.out = nullptr; a.p = 0;
    a.ep_x = xs; a.ep_x_stride = (long)hX;
    a.ep_p = pv; a.ep_p_stride = (long)hP;
    a.ep_r = rv; a.ep_r_stride = (long)hP;
    a.red = h->red_args(FIN_BETA, MODE_RUN);
    RK(h->run_hop(h->hop_launch(lat, P, HOP_P2, 1, EPI_CG, nrhs), a, s));
    KL(cg_update_p(P, pv, rv, Vh, (long)hP, nrhs, h->cg_dev, s, hist, hcap));
    return OQ_OK;
  };

  // The intermediate resets of a low-precision solve use double-float
  // arithmetic (OQ_OPT_DF64_RESETS, default; else binary64 as in the
  // paper); every convergence decision is still taken in binary64.
  // A binary64 phase resets in binary64 (its inner solve reaches the target).
  bool df_ok = h->df64_resets;
  auto reset_prec_of = [&]() { return (P != P_F64 && df_ok) ? P_DF64 : P_F64; };
  // steps of each rhs at the start of its current inner solve, and the
  // length of its previous inner solve (0: none yet)
  std::vector<int> inner_start(nrhs, 0), inner_len(nrhs, 0);
  auto mark_starts = [&]() {
    for (int k = 0; k < nrhs; ++k)
      if (cs[k].mode == MODE_RESET) inner_start[k] = cs[k].steps;
  };
  int pending = decide(false);
  mark_starts();
  RK(upload());
  if (pending) RK(restart());
  for (;;) {
    RK(download());
    int run = 0, rst = 0, park = 0;
    for (int k = 0; k < nrhs; ++k) {
      run += cs[k].mode == MODE_RUN;
      rst += cs[k].mode == MODE_RESET;
      park += cs[k].mode == MODE_PARK;
    }
    if (!run && !rst && park) {
      // every live rhs waits for the next type: advance the phase and decide
      // again for the parked ones (they may skip further phases)
      for (int k = 0; k < nrhs; ++k) {
        phase_steps[4 * k + phase] = cs[k].steps - steps_before[k];
        steps_before[k] = cs[k].steps;
      }
      phase += 1;
      P = phase_prec[phase];
      XP = P == P_F64 ? P_F64 : P_F32;
      hP = spinor_half_bytes(Vh, P);
      hX = spinor_half_bytes(Vh, XP);
      set_phase_args();
      int fmt = -1;
      bool mixed = false;
      for (int k = 0; k < nrhs; ++k)
        if (cs[k].mode == MODE_PARK) {
          cs[k].mode = MODE_RESET;
          mixed |= fmt >= 0 && rd_fmt[k] != fmt;
          fmt = rd_fmt[k];
        }
      if (mixed) {
        // a binary64 confirmation reset some of them after others were parked:
        // recompute every parked residual in binary64 (x_d unchanged)
        RK(upload());
        RK(reset_step(P_F64, false));
        RK(download());
      }
      pending = decide(false);
      mark_starts();
      RK(upload());
      if (pending) RK(restart());
      continue;
    }
    if (rst) {
      for (int k = 0; k < nrhs; ++k)
        if (cs[k].mode == MODE_RESET) inner_len[k] = cs[k].steps - inner_start[k];
      int reset_prec = reset_prec_of();
      // a reset whose inner solves all stopped on the target (their recursive
      // residual claims convergence) is the one expected to end the solve: it
      // is computed in binary64 directly instead of double-float followed by
      // the binary64 confirmation
      if (reset_prec == P_DF64) {
        bool all_tol = true;
        for (int k = 0; k < nrhs; ++k)
          if (cs[k].mode == MODE_RESET && cs[k].reason != WHY_TOL) all_tol = false;
        if (all_tol) reset_prec = P_F64;
      }
      RK(reset_step(reset_prec, true));
      RK(download());
      if (reset_prec == P_DF64) {
        // a double-float residual may only propose convergence: confirm it with
        // binary64 arithmetic before deciding (and keep binary64 from then on if
        // the double-float value was too optimistic)
        bool claims = false;
        for (int k = 0; k < nrhs; ++k)
          if (cs[k].mode == MODE_RESET && sqrt(cs[k].rd2) <= prm->res * eta_n[k]) claims = true;
        if (claims) {
          std::vector<double> df(nrhs);
          for (int k = 0; k < nrhs; ++k) df[k] = cs[k].rd2;
          RK(reset_step(P_F64, false));
          RK(download());
          for (int k = 0; k < nrhs; ++k)
            if (cs[k].mode == MODE_RESET && sqrt(df[k]) <= prm->res * eta_n[k] &&
                sqrt(cs[k].rd2) > prm->res * eta_n[k])
              df_ok = false;
        }
      }
      if (hist)
        for (int k = 0; k < nrhs; ++k)
          if (cs[k].mode == MODE_RESET) {
            reset_hist[k].push_back((double)cs[k].steps);
            reset_hist[k].push_back(eta_n[k] > 0.0 ? sqrt(cs[k].rd2) / eta_n[k] : 0.0);
          }
      pending = decide(true);
      mark_starts();
      RK(upload());
      if (pending) RK(restart());
      continue;
    }
    if (!run) break;
    int chunk = CHUNK;
    for (int k = 0; k < nrhs; ++k) {
      if (cs[k].mode != MODE_RUN || inner_len[k] == 0) continue;
      int left = inner_len[k] - 1 - (cs[k].steps - inner_start[k]);
      left = left < 1 ? 1 : left;
      chunk = left < chunk ? left : chunk;
    }
    for (int k = 0; k < chunk; ++k) RK(iteration());
  }

  // psi = x_d on the even sites, zero on the odd sites (the even-site layout
  // has no odd sites: every entry is written by the unpacking)
  if (!half) CK(cudaMemsetAsync(psi_dev, 0, canon_field * nrhs, s));
  KL(unpack_spinor(L.g, P_F64, OQ_EVEN, xd, psi_dev, 1.0, nrhs, (long)h64, canon_stride, s, half));
  CK(cudaStreamSynchronize(s));
  if (hist) {
    std::vector<double> rec((size_t)hcap * nrhs);
    CK(cudaMemcpy(rec.data(), hist, sizeof(double) * rec.size(), cudaMemcpyDeviceToHost));
    h->hist_rec.assign(nrhs, {});
    for (int k = 0; k < nrhs; ++k) {
      const int m = cs[k].steps < hcap ? cs[k].steps : hcap;
      for (int j = 0; j < m; ++j)
        h->hist_rec[k].push_back(eta_n[k] > 0.0 ? rec[(size_t)k * hcap + j] / eta_n[k] : 0.0);
    }
    h->hist_reset = reset_hist;
    h->hist_nrhs = nrhs;
  }
  int ret = OQ_OK;
  for (int k = 0; k < nrhs; ++k) {
    phase_steps[4 * k + phase] = cs[k].steps - steps_before[k];
    for (int i = 0; i < 4; ++i) st[k].ladder_steps[i] = phase_steps[4 * k + i];
    st[k].steps = cs[k].steps;
    st[k].resets = resets[k];
    st[k].restarts = 0;
    st[k].cycles = 0;
    st[k].mr_avg = 0.0;
    st[k].nn_fallback = 0;
    st[k].true_rel_res = eta_n[k] > 0.0 ? sqrt(cs[k].rd2) / eta_n[k] : 0.0;
    st[k].converged = (isfinite(cs[k].rd2) && st[k].true_rel_res <= prm->res) ? 1 : 0;
    if (!isfinite(cs[k].rd2)) ret = OQ_ERR_NONFINITE;
    else if (!st[k].converged && ret == OQ_OK) ret = OQ_ERR_NOCONV;
  }
  return ret;
#undef CK
#undef RK
#undef KL
}

extern "C" int oq_cgne_solve(oq_handle h, int lat, const oq_solver_params* prm, const double* eta_dev,
                             double* psi_dev, int nrhs, oq_status* st, void* stream) {
  return cgne_impl(h, lat, prm, eta_dev, psi_dev, nrhs, st, stream, 0);
}

extern "C" int oq_cgne_solve_even(oq_handle h, int lat, const oq_solver_params* prm, const double* eta_dev,
                                  double* psi_dev, int nrhs, oq_status* st, void* stream) {
  return cgne_impl(h, lat, prm, eta_dev, psi_dev, nrhs, st, stream, 1);
}
