// The handle behind the C ABI: per-lattice packed gauge/clover state, a
// grow-only workspace of named device buffers, the reduction scratch, the
// per-kernel launch shapes chosen by the tuner, and optional CUDA-event
// timing of every stencil launch.
#pragma once
#include <cuda_runtime.h>
#include <string.h>

#include <map>
#include <string>
#include <vector>

#include "../../include/oq.h"
#include "oq_internal.h"
#include "oq_kernels.h"

namespace oq {

struct DevBuf {
  void* p = nullptr;
  size_t n = 0;
};

struct LatCtx {
  Geom g;
  int link_fmt = -1;
  bool has_gauge = false, has_clover = false;
  double kappa = 0.0, csw = 0.0;
  DevBuf u64, u32, a64, a32, i64, i32;
  DevBuf u32_18;  // 18-real binary32 copy kept next to 12-real links
  // double-float (hi, lo) splits of the binary64 links, clover and inverse
  // clover, made on the first DF64 use after an upload / clover build
  DevBuf udf, adf, idf;
  bool df_ready = false;
  // Schroedinger-functional lattices (bc_t = 0) and QCD+QED uploads keep the
  // unmasked binary64 links the clover is built from (SU(3) part for QCD+QED)
  // and the packed U(1) angles with their charge
  DevBuf uclov, au1;
  bool uclov_valid = false, has_u1 = false;
  // time-split sub-domain (OQ_BC_HALO): its time hops across x0 = 0 / T-1
  // read faces of the neighbouring sub-domains; uext holds the packed binary64
  // links of the sub-domain extended by one slice on each side (clover build)
  bool halo_t = false, has_uext = false;
  // C* boundaries in this many spatial directions (x1 first): the lattice is
  // doubled in x1 (g.L[1] = 2 L1); 0 = none
  int cstar = 0;
  DevBuf uext;
  double qcharge = 0.0, cF = 1.0, csw_qed = 0.0;
  std::map<std::string, DevBuf> ws;
};

// one timed stencil launch: its algorithmic bytes are fixed (links, clover:
// read once if any right-hand side is live) + per_rhs x (live right-hand
// sides), the live count read back from slot `slot` of the device record
struct ProfRec {
  cudaEvent_t e0, e1;
  int mode, epi, prec, nr, link_fmt, dag;
  double fixed, per_rhs;
  int nrhs;
  long slot;  // -1: no record slot (counted as all right-hand sides live)
};

// tuned CTA shape of one stencil variant; epi = EPI_NONE is the entry for
// every epilogue the tuner did not time separately
struct TuneKey {
  int lat, prec, mode, nrhs, epi;
  bool operator<(const TuneKey& o) const {
    if (lat != o.lat) return lat < o.lat;
    if (prec != o.prec) return prec < o.prec;
    if (mode != o.mode) return mode < o.mode;
    if (nrhs != o.nrhs) return nrhs < o.nrhs;
    return epi < o.epi;
  }
};

// the launch shape chosen for one stencil variant (by the tuner or set)
struct TuneVal {
  int bx = 128, by = 1;  // CTA: bx sites x by groups of nr right-hand sides
  int nr = 1;            // right-hand sides per thread
  int regcap = 0;        // register-capped multi-rhs variant
  int link_fmt = -1;     // binary32 link format (-1: the uploaded one)
  float ms = 0.f;        // tuner's time per launch (0 if set by hand)
};

}  // namespace oq

struct oq_ctx {
  int device = 0;
  std::vector<oq::LatCtx> lats;
  // reduction scratch
  double* partials = nullptr;
  size_t partials_n = 0;
  unsigned* counters = nullptr;
  size_t counters_n = 0;
  double* results = nullptr;
  double* results_host = nullptr;  // pinned
  size_t results_n = 0;
  int* status_dev = nullptr;
  oq::CgState* cg_dev = nullptr;
  oq::CgState* cg_host = nullptr;  // pinned mirror
  size_t cg_n = 0;
  // launch shapes
  std::map<oq::TuneKey, oq::TuneVal> tuned;
  // kernels launched by this handle so far
  long long launches = 0;
  // CGNE: intermediate reset residuals in double-float arithmetic (default:
  // ~3x faster per pass than binary64 on GB300; every stop decision binary64)
  bool df64_resets = true;   // OQ_OPT_DF64_RESETS
  // test hook: the tensor-core PTC layer issues no MMA, so its bounded wait runs out
  bool hook_tc_skip_commit = false;
  // SAP block kernel: 0 operands staged in shared memory, 1 operands from
  // global memory, 2 the same register-capped for two CTAs per SM
  int sap_kernel = 0;        // OQ_OPT_SAP_KERNEL
  // NN-preconditioned GCR applies the network with the tensor-core layers
  // instead of the (measured faster) binary32 CUDA-core ones
  bool nn_tensor_cores = false;
  // solver diagnostics (OQ_OPT_HISTORY): CGNE's relative recursive residual
  // after every regular step and its relative residual at every reset, per
  // rhs, of the last solve that recorded them
  bool history = false;
  int hist_nrhs = 0;                                    // 0: nothing recorded
  std::vector<std::vector<double>> hist_rec;            // [rhs][step - 1]
  std::vector<std::vector<double>> hist_reset;          // [rhs]: step, residual, step, residual, ...
  // profiling
  bool prof_on = false;
  std::vector<oq::ProfRec> prof;
  std::vector<cudaEvent_t> event_pool;
  // per profiled launch: right-hand sides live in it (written by the kernel)
  unsigned* prof_live = nullptr;
  size_t prof_live_n = 0;

  int alloc(oq::DevBuf* b, size_t n) {
    if (b->n >= n && b->p) return OQ_OK;
    if (b->p) {
      cudaDeviceSynchronize();
      cudaFree(b->p);
      b->p = nullptr;
      b->n = 0;
    }
    if (cudaMalloc(&b->p, n) != cudaSuccess) {
      cudaGetLastError();
      return OQ_ERR_NOMEM;
    }
    b->n = n;
    return OQ_OK;
  }

  int workspace(int lat, const char* name, size_t n, void** out) {
    oq::DevBuf& b = lats[lat].ws[name];
    int rc = alloc(&b, n);
    *out = b.p;
    return rc;
  }

  // library-owned stream for graph capture and replay (the caller's stream
  // may be the legacy default stream, which cannot be captured)
  cudaStream_t work_stream = nullptr;
  int ensure_work_stream() {
    if (!work_stream && cudaStreamCreateWithFlags(&work_stream, cudaStreamNonBlocking) != cudaSuccess)
      return OQ_ERR_CUDA;
    return OQ_OK;
  }

  // pinned host staging for small coefficient uploads (4 KiB)
  void* stage_host = nullptr;
  int ensure_stage() {
    if (!stage_host && cudaMallocHost(&stage_host, 4096) != cudaSuccess) return OQ_ERR_NOMEM;
    return OQ_OK;
  }

  int ensure_scratch() {
    if (!status_dev && cudaMalloc(&status_dev, 64) != cudaSuccess) return OQ_ERR_NOMEM;
    return OQ_OK;
  }

  // room for `slots` reductions of `grid` partials each
  int ensure_reduce(int slots, long grid) {
    int rc = ensure_scratch();
    if (rc) return rc;
    size_t np = (size_t)slots * (size_t)grid;
    if (np > partials_n) {
      cudaDeviceSynchronize();
      cudaFree(partials);
      partials = nullptr;
      if (cudaMalloc(&partials, np * sizeof(double)) != cudaSuccess) return OQ_ERR_NOMEM;
      partials_n = np;
    }
    if ((size_t)slots > counters_n) {
      cudaDeviceSynchronize();
      cudaFree(counters);
      cudaFree(results);
      cudaFreeHost(results_host);
      counters = nullptr;
      results = nullptr;
      results_host = nullptr;
      size_t n = (size_t)slots < 64 ? 64 : (size_t)slots;
      if (cudaMalloc(&counters, n * sizeof(unsigned)) != cudaSuccess) return OQ_ERR_NOMEM;
      if (cudaMemset(counters, 0, n * sizeof(unsigned)) != cudaSuccess) return OQ_ERR_CUDA;
      if (cudaMalloc(&results, 2 * n * sizeof(double)) != cudaSuccess) return OQ_ERR_NOMEM;
      if (cudaMallocHost(&results_host, 2 * n * sizeof(double)) != cudaSuccess) return OQ_ERR_NOMEM;
      counters_n = n;
      results_n = 2 * n;
    }
    return OQ_OK;
  }

  int ensure_cg(int nrhs) {
    if ((size_t)nrhs <= cg_n) return OQ_OK;
    cudaDeviceSynchronize();
    cudaFree(cg_dev);
    cudaFreeHost(cg_host);
    cg_dev = nullptr;
    cg_host = nullptr;
    if (cudaMalloc(&cg_dev, nrhs * sizeof(oq::CgState)) != cudaSuccess) return OQ_ERR_NOMEM;
    if (cudaMallocHost(&cg_host, nrhs * sizeof(oq::CgState)) != cudaSuccess) return OQ_ERR_NOMEM;
    cg_n = nrhs;
    return OQ_OK;
  }

  oq::RedArgs red_args(int fin, int gate) {
    oq::RedArgs r;
    r.partials = partials;
    r.counters = counters;
    r.result = results;
    r.cg = cg_dev;
    r.fin = fin;
    r.gate = gate;
    return r;
  }

  oq::HopArgs hop_args(int lat, int prec) {
    oq::LatCtx& L = lats[lat];
    oq::HopArgs a;
    memset(&a, 0, sizeof(a));
    a.g = L.g;
    if (prec == oq::P_DF64) {  // ensure_df(lat) has made the splits
      a.links = L.udf.p;
      a.clov = L.adf.p;
      a.cinv = L.idf.p;
    } else {
      const bool f64 = prec == oq::P_F64;
      a.links = f64 ? L.u64.p : L.u32.p;
      a.clov = f64 ? L.a64.p : L.a32.p;
      a.cinv = f64 ? L.i64.p : L.i32.p;
    }
    a.nrhs = 1;
    a.lat = lat;
    return a;
  }

  // the double-float splits of links and clover that DF64 kernels read
  int ensure_df(int lat, cudaStream_t s) {
    oq::LatCtx& L = lats[lat];
    if (L.df_ready) return OQ_OK;
    if (!L.has_clover) return OQ_ERR_STATE;
    const size_t nu = (size_t)2 * 4 * 18 * L.g.Vh, na = (size_t)2 * 72 * L.g.Vh;
    int rc = alloc(&L.udf, nu * sizeof(float2));
    if (!rc) rc = alloc(&L.adf, na * sizeof(float2));
    if (!rc) rc = alloc(&L.idf, na * sizeof(float2));
    if (rc) return rc;
    if (oq::split_f64((const double*)L.u64.p, L.udf.p, nu, s) != cudaSuccess ||
        oq::split_f64((const double*)L.a64.p, L.adf.p, na, s) != cudaSuccess ||
        oq::split_f64((const double*)L.i64.p, L.idf.p, na, s) != cudaSuccess)
      return OQ_ERR_CUDA;
    L.df_ready = true;
    return OQ_OK;
  }

  oq::HopLaunch hop_launch(int lat, int prec, int mode, int dagger, int epi, int nrhs) {
    oq::HopLaunch l;
    l.prec = prec;
    l.link_fmt = lats[lat].link_fmt;
    l.mode = mode;
    l.dagger = dagger;
    l.epi = epi;
    auto it = tuned.find(oq::TuneKey{lat, prec, mode, nrhs, epi});
    if (it == tuned.end()) it = tuned.find(oq::TuneKey{lat, prec, mode, nrhs, oq::EPI_NONE});
    if (it != tuned.end()) {
      l.bx = it->second.bx;
      l.by = it->second.by;
      l.nr = it->second.nr;
      l.regcap = it->second.regcap;
      if (it->second.link_fmt >= 0) l.link_fmt = it->second.link_fmt;
    } else if (nrhs == 1) {
      l.bx = 128;
      l.by = 1;
    } else {
      // several right-hand sides: 32 sites x (largest divisor of nrhs <= 8) rows
      l.bx = 32;
      l.by = 1;
      for (int d = 8; d >= 1; --d)
        if (nrhs % d == 0) {
          l.by = d;
          break;
        }
    }
    if (l.by > nrhs) l.by = nrhs;
    return l;
  }

  // algorithmic bytes of one stencil launch (each operand counted once), as
  // the part read once per launch (links, clover) and the part per live
  // right-hand side (spinors and epilogue vectors)
  void hop_bytes_parts(const oq::HopLaunch& l, const oq::HopArgs& a, double* fixed, double* per_rhs) {
    const double sp = oq::prec_bytes(l.prec);
    const bool wide = l.prec == oq::P_F64 || l.prec == oq::P_DF64;  // binary64 links and clover
    const double su = wide ? 8.0 : 4.0;
    const double ru = (!wide && l.link_fmt == oq::LINK_12) ? 12.0 : 18.0;
    const double sites = (double)a.g.Vh * (l.mode == oq::HOP_DW ? 2.0 : 1.0);
    double spin = 0.0;
    double links = 0.0;
    if (l.mode == oq::HOP_DW) {
      spin = 48.0 * sp;          // in + out
      links = 4.0 * ru * su;     // every link once for the full lattice
    } else {
      spin = (l.mode == oq::HOP_P1 ? 48.0 : 72.0) * sp;
      links = 8.0 * ru * su;     // all links once per half-lattice pass
    }
    if (l.epi == oq::EPI_CG) spin += (24.0 + 24.0 + 48.0 - 24.0) * sp + 48.0 * (l.prec == oq::P_F64 ? 8.0 : 4.0);
    if (l.epi == oq::EPI_RESID64) spin += 24.0 * sp;
    const double clov = 72.0 * su;
    *fixed = sites * (links + clov);
    *per_rhs = sites * spin;
  }

  // all right-hand sides live
  double hop_bytes(const oq::HopLaunch& l, const oq::HopArgs& a) {
    double f = 0.0, r = 0.0;
    hop_bytes_parts(l, a, &f, &r);
    return f + r * a.nrhs;
  }

  // the binary32 link copy that matches the launch's link format
  oq::HopArgs with_links(const oq::HopLaunch& l, const oq::HopArgs& a) {
    oq::HopArgs b = a;
    if (l.prec != oq::P_F64 && l.prec != oq::P_DF64 && a.lat >= 0 && a.lat < (int)lats.size()) {
      const oq::LatCtx& L = lats[a.lat];
      if (l.link_fmt == oq::LINK_18 && L.link_fmt == oq::LINK_12 && L.u32_18.p) b.links = L.u32_18.p;
    }
    return b;
  }

  int run_hop(const oq::HopLaunch& l, const oq::HopArgs& a, cudaStream_t s) {
    oq::ProfRec rec;
    rec.slot = -1;
    if (prof_on) {
      if (event_pool.size() < 2) {
        for (int k = 0; k < 64; ++k) {
          cudaEvent_t e;
          if (cudaEventCreate(&e) != cudaSuccess) return OQ_ERR_CUDA;
          event_pool.push_back(e);
        }
      }
      rec.e1 = event_pool.back();
      event_pool.pop_back();
      rec.e0 = event_pool.back();
      event_pool.pop_back();
      rec.mode = l.mode;
      rec.epi = l.epi;
      rec.prec = l.prec;
      rec.nr = l.nr;
      rec.dag = l.dagger;
      rec.link_fmt = (l.prec == oq::P_F64 || l.prec == oq::P_DF64) ? -1 : l.link_fmt;
      hop_bytes_parts(l, a, &rec.fixed, &rec.per_rhs);
      rec.nrhs = a.nrhs;
      rec.slot = prof.size() < prof_live_n ? (long)prof.size() : -1;
      cudaEventRecord(rec.e0, s);
    }
    oq::HopArgs b = with_links(l, a);
    b.live_rec = (prof_on && rec.slot >= 0) ? prof_live + rec.slot : nullptr;
    cudaError_t e = oq::launch_hop(l, b, s);
    launches += 1;
    if (prof_on) {
      cudaEventRecord(rec.e1, s);
      prof.push_back(rec);
    }
    return e == cudaSuccess ? OQ_OK : OQ_ERR_CUDA;
  }

  void release() {
    for (auto& L : lats) {
      oq::DevBuf* bs[] = {&L.u64, &L.u32, &L.a64, &L.a32, &L.i64, &L.i32, &L.u32_18, &L.udf, &L.adf, &L.idf, &L.uclov, &L.au1,
                          &L.uext};
      for (auto* b : bs) cudaFree(b->p);
      for (auto& kv : L.ws) cudaFree(kv.second.p);
    }
    cudaFree(prof_live);
    cudaFree(partials);
    cudaFree(counters);
    cudaFree(results);
    cudaFreeHost(results_host);
    cudaFree(status_dev);
    cudaFree(cg_dev);
    cudaFreeHost(cg_host);
    cudaFreeHost(stage_host);
    if (work_stream) cudaStreamDestroy(work_stream);
    for (auto& r : prof) {
      cudaEventDestroy(r.e0);
      cudaEventDestroy(r.e1);
    }
    for (auto e : event_pool) cudaEventDestroy(e);
  }
};
