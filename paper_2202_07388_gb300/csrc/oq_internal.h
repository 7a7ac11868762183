// Host/device shared declarations of the library internals (not part of the
// public C ABI in include/oq.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include "oq_device.cuh"

namespace oq {

// Per right-hand-side state of the CGNE solver, resident in device memory so
// that the regular steps never wait for the host.
struct CgState {
  double rr;        // ||r_s||^2 of the small-type residual
  double rr_start;  // ||r_s||^2 at the last (re)start
  double pAp;       // ||Dhat p||^2
  double alpha, beta;
  double tol2;      // stop threshold on rr (scaled units)
  double delta2;    // reset threshold factor delta^2
  double scale;     // s: the small-type system is A x_s = r_d / s
  double rd2;       // ||r_d||^2 of the binary64 residual after a reset
  int mode;         // MODE_RUN, MODE_RESET, MODE_DONE, MODE_PARK
  int reason;       // why regular steps stopped
  int steps;        // regular steps so far
  int nmx;
};
// MODE_PARK: reset, waiting for the next storage type of a precision ladder
// (no kernel acts on it)
enum { MODE_RUN = 0, MODE_RESET = 1, MODE_DONE = 2, MODE_PARK = 3 };
enum { WHY_NONE = 0, WHY_DELTA = 1, WHY_TOL = 2, WHY_NMX = 3, WHY_NONFINITE = 4, WHY_BREAKDOWN = 5 };

// reduction finishers run by the last CTA of a grid reduction
enum Fin : int { FIN_STORE = 0, FIN_ALPHA = 1, FIN_BETA = 2, FIN_RESTART = 3, FIN_RD2 = 4 };

struct RedArgs {
  double* partials;    // [nrhs][gridDim.x]
  unsigned* counters;  // [nrhs]
  double* result;      // [nrhs] (FIN_STORE)
  CgState* cg;         // [nrhs]
  int fin;
  int gate;            // CG finishers act only on rhs with cg[rhs].mode == gate
};

enum HopMode : int { HOP_DW = 0, HOP_P1 = 1, HOP_P2 = 2 };
enum HopEpi : int { EPI_NONE = 0, EPI_NORM = 1, EPI_CG = 2, EPI_RESID64 = 3 };

struct HopArgs {
  Geom g;
  const void* in;      // neighbour field (parity 1-p), packed
  const void* in2;     // site-local field (parity p) for the clover term
  void* out;           // output field (parity p)
  const void* links;   // packed links
  const void* clov;    // packed A
  const void* cinv;    // packed A^{-1}
  long in_stride;      // bytes between right-hand sides
  long in2_stride;
  long out_stride;
  long half_bytes;     // bytes of one packed half field (HOP_DW: parity offset)
  int p;               // output parity (ignored for HOP_DW: blockIdx.z)
  int nrhs;
  int gate;            // run only right-hand sides with cg[rhs].mode == gate (cg != null)
  // epilogue operands (EPI_CG: x += alpha p, r -= alpha q; EPI_RESID64: r = eta - out)
  void* ep_x;
  const void* ep_p;
  void* ep_r;
  const void* ep_eta;
  long ep_x_stride, ep_p_stride, ep_r_stride, ep_eta_stride;
  RedArgs red;
  CgState* cg;
  int lat;             // host side: lattice of the handle these arguments belong to
  // instrumentation (nullable): CTA 0 writes the number of right-hand sides
  // live in this launch (not gated off by their solver state)
  unsigned* live_rec;
  // sub-domain launches (halo_next != null): the time hops that leave the
  // sub-domain read faces (load_half layout) received from the neighbouring
  // sub-domains instead of the periodic wrap: halo_next the projected half
  // spinors (1 -/+ g0) psi of the next one's x0 = 0 slice, halo_prev the
  // transported U_0^dag (1 +/- g0) psi of the previous one's last slice;
  // halo_sign_* the boundary factor of those hops
  const void* halo_next;
  const void* halo_prev;
  long halo_stride;    // bytes between right-hand sides of a face
  long halo_pstride;   // HOP_DW: bytes between the faces of the two output parities
  float halo_sign_next, halo_sign_prev;
};

// the number of right-hand sides a launch acts on, written by one thread of CTA 0
// before the CTA contributes to any reduction (so before any finisher runs)
__device__ __forceinline__ void record_live(const HopArgs& a) {
  if (a.live_rec && blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) {
    unsigned n = 0;
    for (int r = 0; r < a.nrhs; ++r) n += (!a.cg || a.cg[r].mode == a.gate) ? 1u : 0u;
    *a.live_rec = n;
  }
}

struct HopLaunch {
  int prec;      // Prec of in/in2/out
  int link_fmt;  // LINK_18 / LINK_12 (F32/BF16/F16 only)
  int mode;      // HopMode
  int dagger;
  int epi;       // HopEpi
  int bx, by;    // CTA shape: bx sites x by groups of nr right-hand sides
  int nr = 1;    // right-hand sides per thread (1: hop_kernel; 2, 4: hop_mr_kernel)
  int regcap = 0;  // hop_mr_kernel: 1 = register-capped variant
  // batched launch over several systems (hop_batch_kernel) when sys != null:
  // per-system arguments and the (system, site block) tile list in device memory
  const HopArgs* sys = nullptr;
  const int2* tiles = nullptr;
  int ntiles = 0;
  int grid = 0;
};

cudaError_t launch_hop(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
cudaError_t launch_hop_f64(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
cudaError_t launch_hop_f32(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
cudaError_t launch_hop_bf16(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
cudaError_t launch_hop_f16(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
cudaError_t launch_hop_df64(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
// several right-hand sides per thread (binary32 arithmetic types, nr = 2 or 4)
cudaError_t launch_hop_mr2_f32(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
cudaError_t launch_hop_mr4_f32(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
cudaError_t launch_hop_mr2_bf16(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
cudaError_t launch_hop_mr4_bf16(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
cudaError_t launch_hop_mr2_f16(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
cudaError_t launch_hop_mr4_f16(const HopLaunch& L, const HopArgs& a, cudaStream_t s);
// double-float, 2 right-hand sides per thread (packed two-lane arithmetic)
cudaError_t launch_hop_df2(const HopLaunch& L, const HopArgs& a, cudaStream_t s);

// geometry of a sub-domain extended by one time slice on each side
inline Geom halo_ext_geom(const Geom& g) {
  Geom e = g;
  const long Fs = g.Vh / g.L[0];
  e.L[0] = g.L[0] + 2;
  e.Vh = g.Vh + 2 * Fs;
  geom_init_div(e);
  return e;
}

__host__ __device__ inline int prec_bytes(int prec) {
  return (prec == P_F64 || prec == P_DF64) ? 8 : prec == P_F32 ? 4 : 2;
}
__host__ __device__ inline long spinor_half_bytes(long Vh, int prec) { return 24L * Vh * prec_bytes(prec); }

}  // namespace oq
