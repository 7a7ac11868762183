// Host-side launchers of the kernels, shared between translation units.
#pragma once
#include "oq_internal.h"

struct oq_ctx;

namespace oq {

// A (optional): canonical U(1) angles A_mu(x) multiplied into the links as
// exp(i q A); uclov (optional): the packed binary64 links before the phase;
// au1 (optional): the packed angles
// cs_l1 > 0: C* lattice doubled in x1; canon holds the physical links (x1 < cs_l1)
// and the second half gets their complex conjugates (U(1) angles negated)
cudaError_t pack_links(const Geom& g, const double* canon, double* u64, void* u32, int fmt, void* u18,
                       const double* A, double q, double* uclov, double* au1, cudaStream_t s, int cs_l1 = 0);
// Schroedinger-functional boundaries: zero the time-like links of slices
// x0 = 0 and x0 = T-1 in every hopping copy
cudaError_t sf_mask_links(const Geom& g, double* u64, void* u32, int fmt, void* u18, cudaStream_t s);
// half (subset EVEN or ODD only): the canonical field holds the sites of that
// parity only, site-lexicographic index / 2
cudaError_t pack_spinor(const Geom& g, int prec, int subset, const double* canon, void* out, double scale,
                        int nrhs, long canon_stride_d2, long out_stride_bytes, cudaStream_t s, int half = 0);
cudaError_t unpack_spinor(const Geom& g, int prec, int subset, const void* in, double* canon, double scale,
                          int nrhs, long in_stride_bytes, long canon_stride_d2, cudaStream_t s, int half = 0);
// binary64 array of n values -> n double-float (hi, lo) pairs
cudaError_t split_f64(const double* in, void* out, size_t n, cudaStream_t s);
// links: packed binary64 links of the field strength; au1 (optional):
// packed U(1) angles with charge q, used as separate U(1) field strength
// with coefficient csw_qed (qed_split) or multiplied into the links
// (the U(3) clover); cF: Schroedinger-functional boundary coefficient
// (bc_t = 0 lattices)
cudaError_t build_clover(const Geom& g, const double* links, const double* au1, double q, int qed_split,
                         double kappa, double csw, double csw_qed, double cF, double* a64, float* a32,
                         double* i64, float* i32, int* status_dev, cudaStream_t s);

// binary64 reductions over packed half fields of Vh sites per rhs
cudaError_t reduce_norm2(int prec, const void* x, long Vh, long stride_bytes, int nrhs, const RedArgs& ra,
                         cudaStream_t s);
cudaError_t reduce_dot(int prec, const void* x, const void* y, long Vh, long stride_bytes, int nrhs,
                       const RedArgs& ra, cudaStream_t s);
int reduce_grid(long nsites);

// CGNE vector kernels (gated on CgState::mode)
// hist (nullable): [nrhs][hcap] record of sqrt(rr) * scale after every regular step
cudaError_t cg_update_p(int prec, void* p, const void* r, long Vh, long stride, int nrhs, const CgState* cg,
                        cudaStream_t s, double* hist = nullptr, int hcap = 0);
// xdf (optional): also write the double-float split of the new x_d (rhs in MODE_RESET)
cudaError_t cg_accumulate_x(int xprec, double* xd, const void* xs, long Vh, long stride_xd, long stride_xs,
                            int nrhs, const CgState* cg, cudaStream_t s,
                            void* xdf = nullptr);
cudaError_t cg_restart(int prec, const void* rd, int rd_prec, void* rs, void* p, void* xs, int xprec, long Vh,
                       long stride_d, long stride_s, long stride_xs, int nrhs, const RedArgs& ra, cudaStream_t s);
// y = a_k x + b_k y per right-hand side (binary64 or binary32 fields of n reals each)
cudaError_t axpby(int prec, const double* a, const void* x, const double* b, void* y, long n, int nrhs,
                  cudaStream_t s);
cudaError_t cg_copy_gated(double* dst, const double* src, long n16, long stride, int nrhs, const CgState* cg,
                          int gate, cudaStream_t s);

// learned preconditioner (ptc.cu): round the binary32 master weights to the
// bfloat16 forward weights held by the handle, and apply M = L2 L1
int nnprec_prepare(struct ::oq_ctx* h, int lat, const float* master, cudaStream_t s);
int nnprec_forward(struct ::oq_ctx* h, int lat, const void* r, void* y, cudaStream_t s);
// the same with the channel contraction on the tensor cores (tcgen05);
// takes the binary32 master weights, synchronises s, OQ_ERR_TIMEOUT on a failed wait
int nnprec_forward_tc(struct ::oq_ctx* h, int lat, const float* master, const void* r, void* y, cudaStream_t s);

// one SAP half cycle: every block of `colour` (binary32 fields); eo: MR on
// the blocks' even-odd Schur complements (needs clov_inv and blocks whose
// operands fit in shared memory, else cudaErrorInvalidValue)
cudaError_t sap_colour(const Geom& g, const int bs[4], int colour, int fmt, const void* links, const void* clov,
                       const void* clov_inv, const void* rho, void* phi, int nmr, int adaptive, float alpha,
                       double tol, unsigned* mr_steps, int kernel, int eo, cudaStream_t s);
size_t sap_smem_bytes(const int bs[4]);

}  // namespace oq
