/*
 * oq: Wilson-clover Dirac operator and mixed-precision solvers for NVIDIA
 * GB300 (sm_103a).  C ABI.
 *
 * The operator is the O(a)-improved Wilson-Dirac operator named in Sec. 1 of
 * Gruber et al., "Performance optimizations for porting the openQ*D package
 * to GPUs" (LATTICE2021), whose application to a spinor field is the
 * SpMV-like kernel the paper singles out (Sec. 1, footnote 1):
 *
 *   (D psi)(x) = A(x) psi(x) - 1/2 sum_mu [ U_mu(x)(1 - g_mu) psi(x+mu)
 *                                        + U_mu(x-mu)^dag (1 + g_mu) psi(x-mu) ]
 *   A(x) = (4 + m0) + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x),  m0 = 1/(2 kappa) - 4,
 *
 * chiral gamma basis (g5 = diag(1,1,-1,-1)), clover-leaf F_{mu nu}, fermion
 * fields antiperiodic (or periodic) in time.  Sites are ordered even-first
 * (Sec. 3, Fig. 3); the even-odd reduced operator is
 *   Dhat = D_ee - D_eo D_oo^{-1} D_oe.
 *
 * Conventions for every entry point:
 *  - Return value: OQ_OK (0) or a negative OQ_ERR_* code; oq_error_string()
 *    names it.  On error nothing was enqueued unless the code is OQ_ERR_CUDA.
 *  - Pointers named *_dev are device pointers owned by the caller; the
 *    library never frees or keeps them beyond the call.  Derived state
 *    (packed links, clover blocks, solver work vectors) is owned by the
 *    handle and freed by oq_destroy().
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Operator applications and packing are asynchronous on it;
 *    the solvers synchronise it before returning (they fill oq_status).
 *  - A handle is used by one host thread at a time.
 *
 * Canonical host layout (binary64 complex, interleaved re/im):
 *   site x = ((x0*L1 + x1)*L2 + x2)*L3 + x3, x0 = time (slowest);
 *   links   U[x][mu][a][b]       (mu = 0..3, 18 doubles per link)
 *   spinors psi[x][spin][colour] (24 doubles per site)
 * Packed device layout (what oq_dw_apply / oq_dw_hat_apply read and write):
 *   one half field per parity, Vh = V/2 sites, eo index = x >> 1, each site's
 *   24 reals in 16-byte chunks stored chunk-major ([chunk][Vh]); F64: 12
 *   chunks, F32: 6 chunks, BF16/F16: 3 chunks.  A full field is the even half
 *   followed by the odd half.  nrhs fields are consecutive in memory.
 *   oq_spinor_bytes() gives the sizes.
 */
#ifndef OQ_H
#define OQ_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct oq_ctx* oq_handle;

/* storage precision of spinor fields (arithmetic is binary32 for F32/BF16/F16).
 * OQ_DF64: double-float storage and arithmetic: every real is an unevaluated
 * sum hi + lo of two binary32 numbers (~48 significant bits), stored as the
 * pair (hi, lo) in 8 bytes (the OQ_F64 sizes; one complex per 16-byte chunk:
 * re.hi, re.lo, im.hi, im.lo), with arithmetic on the binary32 pipes.
 * Accepted by oq_dw_apply, oq_dw_hat_apply, oq_autotune and the packing
 * calls (packing splits binary64 values, unpacking returns hi + lo); the
 * kernels read double-float splits of the links and clover blocks that the
 * handle makes from the binary64 ones on first use; the CGNE uses it for
 * intermediate reset steps (OQ_OPT_DF64_RESETS). */
enum { OQ_F64 = 0, OQ_F32 = 1, OQ_BF16 = 2, OQ_F16 = 3, OQ_DF64 = 4 };
/* storage of the binary32 link copy: 18 reals, or 12 reals with the third
 * row rebuilt as conj(row0 x row1) (SU(3) links only) */
enum { OQ_LINK_18 = 0, OQ_LINK_12 = 1 };
/* field subsets for packing */
enum { OQ_EVEN = 0, OQ_ODD = 1, OQ_FULL = 2 };

enum {
  OQ_OK = 0,
  OQ_ERR_ARG = -1,       /* invalid argument (null pointer, size, enum) */
  OQ_ERR_CUDA = -2,      /* a CUDA call failed */
  OQ_ERR_NOMEM = -3,     /* device allocation failed */
  OQ_ERR_TIMEOUT = -4,   /* a bounded device-side wait gave up */
  OQ_ERR_NONFINITE = -5, /* NaN/Inf met in a binary64 norm */
  OQ_ERR_NOCONV = -6,    /* solver stopped at nmx without reaching res */
  OQ_ERR_STATE = -7      /* call out of order (e.g. no gauge field uploaded) */
};

typedef struct {
  int L[4];  /* L[0] = T, all extents even and >= 2 */
  int bc_t;  /* time boundary: -1 antiperiodic, +1 periodic (the fermion factor of a hop
                across x0 = T-1 <-> 0), or 0 = Schroedinger functional (openQCD boundary
                type 1, Sec. 2 footnote): quark fields vanish at x0 = 0 and x0 = T,
                or OQ_BC_HALO: a time-split sub-domain (see oq_face_pack) */
  int cstar; /* C* boundary conditions in this many spatial directions (0 = periodic; 1: x1;
                2: x1, x2; 3: x1, x2, x3), in the orbifold form of openQ*D (Sec. 1): the
                library's lattice is doubled in x1 (extent 2 L[1]; its fields, canonical
                or packed, have that extent), the second half carrying the
                charge-conjugate copy of the gauge field (oq_gauge_upload takes the
                physical links, of extent L[1], and stores their complex conjugates
                there, U(1) angles negated); a hop across the x2 or x3 boundary of a
                C* direction also moves x1 by L[1].  L[1] must be even. */
} oq_lattice;

/* bc_t of a sub-domain of a lattice split along time (Sec. 3: the lattice is
 * divided into local lattices, one per process).  Its hops across x0 = 0 and
 * x0 = T-1 read faces received from the neighbouring sub-domains; the whole-
 * lattice operators and solvers reject it (OQ_ERR_STATE). */
#define OQ_BC_HALO 2

/* Solver settings, after Table 2 of the paper (res, nmx, nkv, ncy, nmr, bs)
 * plus the storage type of the "small" vectors (sdtype; the "large" type and
 * the reduction type are always binary64, Sec. 2.1, 3.1). */
typedef struct {
  double res;        /* target relative residual (binary64) */
  int nmx;           /* max regular CG steps / GCR steps */
  int nkv;           /* GCR: Krylov vectors before a restart */
  int ncy;           /* SAP cycles per GCR step (maximum if adaptive) */
  int nmr;           /* MR steps per block and cycle (maximum if adaptive) */
  int bs[4];         /* SAP block extents */
  int sdtype;        /* OQ_F64 / OQ_F32 / OQ_BF16 / OQ_F16 */
  double delta;      /* CGNE reset when ||r_rec|| <= delta ||r_reset||; <= 0: 10 eps of sdtype (max 0.1) */
  int adaptive;      /* SAP: adaptive cycle / MR counts (Sec. 3.2) */
  double alpha;      /* SAP adaptive MR ratio threshold (Sec. 3.2, default 0.9) */
  /* CGNE precision ladder (Sec. 2, after Fig. 4): nladder = 0 (zero-initialised
   * struct) runs every regular step in sdtype.  nladder in 1..4: the storage
   * types ladder[0..nladder-1] (each OQ_F64 / OQ_F32 / OQ_BF16 / OQ_F16) replace
   * sdtype; the regular steps of a right-hand side move from ladder[i] to
   * ladder[i+1] at the first reset whose binary64 relative residual is
   * <= ladder_c * eps(ladder[i]) (eps = 2^-10 / 2^-7 / 2^-23 for binary16 /
   * bfloat16 / binary32; ladder_c <= 0 means 1), and delta follows the
   * current type when it is <= 0.  oq_cgne_solve only (the batch: OQ_ERR_ARG). */
  int nladder;
  int ladder[4];
  double ladder_c;
  int sap_eo;        /* SAP block solver: 0 = MR on the block operator D_i; 1 = MR on the block's
                        even-odd Schur complement A_ee - D_eo A_oo^-1 D_oe, odd sites solved
                        exactly afterwards (openQCD's block solver, Sec. 3); needs bs[3] even */
} oq_solver_params;

typedef struct {
  int steps;           /* regular CG steps or GCR steps ("status" of the paper) */
  int resets;          /* CGNE reset steps (binary64 residual recomputations) */
  int restarts;        /* GCR restarts */
  int converged;       /* 1 if true_rel_res <= res */
  double true_rel_res; /* binary64 ||eta - A psi|| / ||eta|| at exit */
  int cycles;          /* SAP-GCR: Schwarz cycles run in total */
  double mr_avg;       /* SAP-GCR: mean MR steps per block solve */
  int ladder_steps[4]; /* CGNE: regular steps run in each storage type of the
                          precision ladder (ladder[i]; index 0 = sdtype without one) */
  int nn_fallback;     /* oq_nn_gcr_solve: 1 if a restart cycle with the network did not halve
                          the residual and SAP (or no preconditioner) took over */
} oq_status;

/* Create a handle for nlat lattices (nlat > 1: an uneven batch).  Selects no
 * device: the current CUDA device at creation is used for every call.
 * Every extent must be even and >= 2, bc_t +1, -1, 0 or OQ_BC_HALO, and the volume at most
 * 2^29 sites (half volume <= 2^28, so site offsets fit 32-bit arithmetic);
 * otherwise OQ_ERR_ARG. */
int oq_create(oq_handle* h, const oq_lattice* lats, int nlat);
int oq_destroy(oq_handle h);
const char* oq_error_string(int code);

/* Bytes of one packed spinor field of lattice `lat` (subset OQ_EVEN/OQ_ODD:
 * half field, OQ_FULL: full field). */
size_t oq_spinor_bytes(oq_handle h, int lat, int prec, int subset);

/* Upload links (canonical binary64 layout, device memory) and build the
 * packed binary64 copy and the binary32 copy in `link_fmt`.  OQ_LINK_12 needs
 * det U = 1 (SU(3)); U(3) = SU(3) x U(1) links need OQ_LINK_18.  Sec. 1
 * (QCD+QED with O(a)-improved Wilson fermions). */
int oq_gauge_upload(oq_handle h, int lat, const double* U_dev, int link_fmt, void* stream);

/* QCD+QED upload (Sec. 1; openQ*D): U_dev the SU(3) links (canonical), A_dev
 * the U(1) potential A_mu(x) (canonical: site-lexicographic, then mu; 4 V
 * binary64 values, device memory) and q the charge.  The hopping term uses
 * the U(3) links U_mu(x) exp(i q A_mu(x)) (18-real binary32 copy); the SU(3)
 * links and the angles are kept for oq_clover_build_ex. */
int oq_gauge_upload_qed(oq_handle h, int lat, const double* U_dev, const double* A_dev, double q,
                        void* stream);

/* Schroedinger-functional lattices (bc_t = 0): the hopping copies of the
 * time-like links of slices x0 = 0 and x0 = T-1 are zero (no hop reaches
 * the x0 = 0 slice), the clover is built from the links as uploaded (the
 * spatial links of slice 0 are the boundary field at x0 = 0 and, by
 * periodicity, at x0 = T), and oq_spinor_pack sets the x0 = 0 slice to zero.
 * Every operator and solver then maps fields that vanish at x0 = 0 to fields
 * that vanish there, as the quark fields of openQCD boundary type 1. */

/* Clover term A(x) and A^{-1}(x) (odd sites) from the uploaded links:
 * clover-leaf field strength, two Hermitian 6x6 chiral blocks per site,
 * built and inverted in binary64, stored in binary64 and binary32.
 * A(x) = 4 + m0 + c_sw (i/4) sum sigma_{mu nu} F_{mu nu}(x), m0 = 1/(2 kappa) - 4;
 * after oq_gauge_upload_qed, F is that of the U(3) links.  Singular block:
 * OQ_ERR_NONFINITE. */
int oq_clover_build(oq_handle h, int lat, double kappa, double csw, void* stream);

typedef struct {
  double kappa;    /* hopping parameter, 4 + m0 = 1/(2 kappa) */
  double csw;      /* coefficient of the SU(3) (or, without qed_split, U(3)) field strength */
  double cF;       /* Schroedinger-functional boundary coefficient: 4 + m0 + cF - 1 at
                      x0 = 1 and x0 = T-1 (bc_t = 0 lattices; 1 = none; ignored otherwise) */
  double csw_qed;  /* qed_split: coefficient of the U(1) field strength of exp(i q A) */
  int qed_split;   /* 1: c_sw F^{SU(3)} + c_sw^QED F^{U(1)} 1_colour (needs oq_gauge_upload_qed);
                      0: c_sw F of the hopping links (U(3) after oq_gauge_upload_qed) */
} oq_clover_params;

/* oq_clover_build with the boundary coefficient c_F of Schroedinger-functional
 * lattices and the separate QED clover coefficient of openQ*D.  qed_split
 * without oq_gauge_upload_qed: OQ_ERR_STATE. */
int oq_clover_build_ex(oq_handle h, int lat, const oq_clover_params* p, void* stream);

/* Convert canonical binary64 spinors (device) to packed `prec` fields and
 * back.  pack multiplies by `scale` before rounding (round to nearest even),
 * unpack divides by it.  subset OQ_EVEN / OQ_ODD read/write only those sites
 * of the canonical field (unpack leaves the other sites untouched); the
 * canonical buffer holds nrhs full-lattice fields either way (V sites x 24
 * doubles each, V = L0 L1 L2 L3), and the packed buffer the size
 * oq_spinor_bytes gives for the subset.  Neither size can be checked here:
 * a shorter buffer is read or written past its end. */
int oq_spinor_pack(oq_handle h, int lat, int prec, int subset, const double* canon_dev,
                   void* packed_dev, double scale, int nrhs, void* stream);
int oq_spinor_unpack(oq_handle h, int lat, int prec, int subset, const void* packed_dev,
                     double* canon_dev, double scale, int nrhs, void* stream);

/* out = D in (dagger: D^dag in = g5 D g5 in) on full packed fields of
 * precision prec (Sec. 1, footnote 1).  in and out must not overlap. */
int oq_dw_apply(oq_handle h, int lat, int prec, const void* in_dev, void* out_dev, int nrhs,
                int dagger, void* stream);

/* out_e = Dhat in_e (or Dhat^dag), even half fields of precision prec
 * (Sec. 3, Fig. 3 even-odd ordering).  Two passes; the odd intermediate
 * lives in handle-owned scratch.  in and out must not overlap. */
int oq_dw_hat_apply(oq_handle h, int lat, int prec, const void* in_dev, void* out_dev, int nrhs,
                    int dagger, void* stream);

/* Same result as oq_dw_hat_apply, for callers that cannot allocate device
 * memory.  No counterpart in the paper: this is a service of the library.
 *
 * oq_dw_hat_apply keeps its odd-site intermediate in handle-owned scratch
 * that it allocates with cudaMalloc the first time it needs more (and growing
 * it synchronises the device).  Some callers cannot allow that: a host
 * program that hands out all device memory through its own pool allocator
 * and forbids allocations behind its back, or one that must keep a fixed
 * device-memory footprint once it has started.  This variant allocates
 * nothing: the intermediate lives in one file-scope device array of
 * OQ_NOALLOC_SCRATCH_BYTES (16 MiB), which every GPU that loads the library
 * holds until the process exits.  The caller still passes the input and
 * output fields (packed even half fields, as for oq_dw_hat_apply) and the
 * handle must already hold the gauge field and clover term.
 *  - prec is OQ_F64, OQ_F32, OQ_BF16 or OQ_F16.  OQ_DF64 is rejected
 *    (OQ_ERR_ARG, nothing enqueued): its kernels read double-float splits of
 *    the links and clover that the handle allocates on their first use.
 *  - The device that is current at the call must be the handle's device,
 *    else OQ_ERR_STATE and nothing is enqueued (the array is per device).
 *  - nrhs * oq_spinor_bytes(h, lat, prec, OQ_EVEN) must not exceed
 *    OQ_NOALLOC_SCRATCH_BYTES, else the call returns OQ_ERR_ARG and enqueues
 *    nothing (binary32: up to 174,762 even sites for one right-hand side).
 *  - Its two stencil launches are timed by oq_profile_start/stop like those
 *    of oq_dw_hat_apply (the profile's records live on the host and in a
 *    buffer that oq_profile_start allocates).
 *  - The first call made while a given device is current looks up the
 *    array's device address on that device (cudaGetSymbolAddress); make that
 *    first call before any stream capture.
 *  - Every call, from any handle, uses the same array, and the array keeps
 *    the last call's contents (each call overwrites what it reads, so nothing
 *    needs clearing).  Calls that overlap on the GPU (e.g. on two streams at
 *    once) race on it: order them on one stream or with events. */
#define OQ_NOALLOC_SCRATCH_BYTES (16u * 1024u * 1024u)
int oq_dw_hat_apply_noalloc(oq_handle h, int lat, int prec, const void* in_dev, void* out_dev, int nrhs,
                            int dagger, void* stream);

/* Autotuner (no counterpart in the paper): time every admissible launch of
 * the full Dw and of both Dhat passes for this (lattice, precision, nrhs) on
 * handle-owned scratch fields with CUDA events, and keep the fastest per pass
 * in the handle; every later stencil launch of that variant, including those
 * inside the solvers, uses it.  Synchronises `stream`.  A launch is: the CTA
 * shape (bx sites x by rows, bx a multiple of 32), the right-hand sides per
 * thread nr (1; or 2, 4 for F32/BF16/F16 storage with nrhs >= nr: the links,
 * clover blocks and indices of a site are loaded once for nr right-hand sides
 * and the arithmetic runs on packed pairs of them; bx*by <= 128), a register
 * cap (regcap 0/1) of the nr > 1 kernels and of the OQ_DF64 kernel (bx*by <=
 * 128; regcap 1: at most 128 registers per thread, 2: at most 168), for the
 * nr > 1 kernels regcap 2: the cap of 1 with each hop's neighbour spinors and
 * link copied ahead into shared memory while the previous hop is computed
 * (12-real links only), regcap 3 (nr = 2): the staged kernel of regcap 2
 * capped at 168 registers instead of 128, and for
 * binary32-arithmetic kernels
 * on 12-real links the 18-real copy the handle keeps (fewer instructions,
 * more bytes).  oq_tune_get reports the chosen launch and its time
 * (link_fmt, nr, regcap nullable; mode 0 = Dw, 1 = Dhat pass 1, 2 = Dhat
 * pass 2); OQ_ERR_STATE if none is set.  The autotuner times pass 2 once per
 * epilogue (they differ in registers and bytes): oq_tune_get_epi reports the
 * launch of one (epi 0 = store, 1 = store and squared norm, 2 = the CGNE
 * update of x and r; OQ_ERR_ARG otherwise), or the mode's plain launch where
 * the epilogue has none of its own (what runs then); oq_tune_get is epi 0.
 * oq_tune_set pins a launch without
 * timing (link_fmt -1: the uploaded format; OQ_ERR_ARG for an inadmissible
 * launch, OQ_ERR_STATE before oq_gauge_upload). */
int oq_autotune(oq_handle h, int lat, int prec, int nrhs, void* stream);
int oq_tune_get(oq_handle h, int lat, int prec, int mode, int nrhs, int* bx, int* by, float* ms,
                int* link_fmt, int* nr, int* regcap);
int oq_tune_get_epi(oq_handle h, int lat, int prec, int mode, int epi, int nrhs, int* bx, int* by, float* ms,
                    int* link_fmt, int* nr, int* regcap);
int oq_tune_set(oq_handle h, int lat, int prec, int mode, int nrhs, int bx, int by, int nr, int regcap,
                int link_fmt);

/* Handle options (no counterpart in the paper).
 * OQ_OPT_DF64_RESETS: 1 (default) = the intermediate CGNE reset steps of a
 *   low-precision solve recompute the residual with OQ_DF64 arithmetic; a
 *   residual that meets the target is confirmed by a binary64 reset before
 *   the solve stops (so the reported true residual, and the stop decision,
 *   are binary64), and a double-float value found too optimistic switches the
 *   solve to binary64 resets.  A reset whose inner solves all stopped on the
 *   target (the recursive residual claims convergence) runs in binary64 at
 *   once.  0 = every reset in binary64 (the paper's
 *   scheme).  On GB300, whose binary64 rate is 1/64 of its binary32 rate, a
 *   double-float reset pass is ~3x faster than a binary64 one.
 * OQ_OPT_TEST_TC_SKIP_MMA: testing aid for failure detection; 1 = the
 *   tensor-core PTC layer issues no MMA, so its bounded (1 s) wait for the
 *   tensor core runs out and oq_nnprec_apply_tc returns OQ_ERR_TIMEOUT with
 *   the device still usable.  Default 0. */
/* OQ_OPT_NN_TENSOR_CORES: 1 = oq_nn_gcr_solve applies the network with the
 *   tensor-core layers of oq_nnprec_apply_tc; default 0 = the binary32
 *   CUDA-core layers of oq_nnprec_apply (measured faster on GB300 for this
 *   small network). */
/* OQ_OPT_SAP_KERNEL: the SAP block kernel (one CTA per block, one thread per
 *   block site).  0 (default) = the block's links (18 reals) and clover
 *   blocks are staged in shared memory once and the MR steps read only shared
 *   memory (falls back to 2 when they do not fit in 227 KB); 1 = operands from
 *   global memory, ~217 registers, one 256-site block per SM; 2 = operands
 *   from global memory, registers capped so that two blocks run per SM.
 *   Other values: OQ_ERR_ARG. */
/* OQ_OPT_HISTORY: 1 = the CGNE solves (oq_cgne_solve, oq_cgne_solve_even)
 *   record solver diagnostics for oq_solve_history; default 0.  Recording
 *   costs one store per right-hand side and regular step. */
enum { OQ_OPT_DF64_RESETS = 1, OQ_OPT_TEST_TC_SKIP_MMA = 2, OQ_OPT_NN_TENSOR_CORES = 3, OQ_OPT_SAP_KERNEL = 4,
       OQ_OPT_HISTORY = 5 };
int oq_set_option(oq_handle h, int key, int value);

/* Solver diagnostics of the last CGNE solve run with OQ_OPT_HISTORY 1
 * (Sec. 2, Fig. 4: the recursive residual of the regular steps against the
 * exact residual of the reset steps), right-hand side rhs:
 *   kind 0: the relative recursive residual ||r_rec|| / ||eta|| after regular
 *     step k at out_host[k-1], k = 1 .. steps (the small-type residual norm
 *     times the inner solve's scale; steps beyond 100,000 are not recorded);
 *   kind 1: every reset step as a pair out_host[2j] = regular steps done
 *     before it, out_host[2j+1] = ||eta - Dhat^dag Dhat x|| / ||eta|| from
 *     the reset's residual (binary64; double-float for an intermediate
 *     double-float reset that did not meet the target).
 * Copies min(cap, available) doubles into out_host (host memory) and sets *n
 * to the number of steps (kind 0) or resets (kind 1) recorded.  OQ_ERR_STATE
 * if no solve recorded any; OQ_ERR_ARG for rhs or kind out of range. */
int oq_solve_history(oq_handle h, int rhs, int kind, double* out_host, int cap, int* n);

/* Binary64 reductions over packed fields: out[k] = ||x_k||^2, and
 * out[2k], out[2k+1] = Re, Im <x_k, y_k> (host arrays of nrhs / 2 nrhs). */
int oq_norm2(oq_handle h, int lat, int prec, int subset, const void* x_dev, int nrhs,
             double* out_host, void* stream);
int oq_dot(oq_handle h, int lat, int prec, int subset, const void* x_dev, const void* y_dev,
           int nrhs, double* out_host, void* stream);

/* ---- Time-split sub-domains (Sec. 3: one local lattice per process) ----
 *
 * A lattice of global extent T x L1 x L2 x L3 split along time into R parts
 * of T_loc = T / R slices (T_loc even) is handled as R sub-domain lattices
 * (bc_t = OQ_BC_HALO, extents T_loc x L1 x L2 x L3; even-odd parities of the
 * sub-domain are the global ones since T_loc is even).  Every application of
 * the operator exchanges two faces per sub-domain and output parity, 12 reals
 * per boundary site (the spin projection halves the spinor):
 *   to_prev: (1 -/+ g0) psi on the sub-domain's x0 = 0 slice, which the
 *            previous sub-domain's forward time hops from its last slice read;
 *   to_next: U_0(x)^dag (1 +/- g0) psi(x) on the x0 = T_loc-1 slice, which the
 *            next sub-domain's backward time hops from its first slice read
 *            (the link lives on the sender, so the sender applies it);
 * (upper signs for Dw, lower for the adjoint).  A face of one parity and one
 * right-hand side is oq_face_bytes(): L1 L2 L3 / 2 sites of 6 complex numbers
 * in the arithmetic type (binary64 for OQ_F64, binary32 for OQ_F32 / BF16 /
 * F16), 16-byte chunks stored chunk-major.  Moving the faces between
 * sub-domains (device copies, NCCL or any transport) is the caller's; the
 * library packs and consumes them.  OQ_DF64 has no sub-domain form. */

/* Links of a sub-domain: U_ext_dev holds the canonical binary64 links of
 * T_loc + 2 time slices (global slices t0 - 1, t0, ..., t0 + T_loc, periodic
 * in the global lattice), so that the clover term of every interior site
 * has all its plaquette leaves.  The hopping term uses the interior slices;
 * oq_clover_build then builds the clover on the extended lattice and keeps
 * the interior (plain c_sw; cF and the QED split are rejected).  OQ_ERR_STATE
 * unless the lattice was created with bc_t = OQ_BC_HALO. */
int oq_gauge_upload_halo(oq_handle h, int lat, const double* U_ext_dev, int link_fmt, void* stream);

/* Bytes of one face (one output parity, one right-hand side); 0 for an
 * invalid lattice or precision (OQ_DF64 included). */
size_t oq_face_bytes(oq_handle h, int lat, int prec);

/* Pack the two faces of packed input fields for their neighbours (see above).
 * subset OQ_EVEN / OQ_ODD: in_dev holds nrhs half fields of that parity and
 * the faces serve the output parity 1 - subset: face k of to_prev_dev /
 * to_next_dev at k * oq_face_bytes().  subset OQ_FULL: in_dev holds full
 * fields and the faces of output parity p are at (p * nrhs + k) *
 * oq_face_bytes().  dagger selects the adjoint's projectors.  Asynchronous. */
int oq_face_pack(oq_handle h, int lat, int prec, int subset, const void* in_dev, int nrhs, int dagger,
                 void* to_prev_dev, void* to_next_dev, void* stream);

/* The faces a sub-domain received: from_next = the next sub-domain's to_prev,
 * from_prev = the previous one's to_next (device pointers, the layout of
 * oq_face_pack), and the boundary factor of the hops across each face (+1, or
 * -1 on the global antiperiodic time boundary: the hop from x0 = T-1 of the
 * last sub-domain to x0 = 0 of the first, and back). */
typedef struct {
  const void* from_next;
  const void* from_prev;
  double sign_next, sign_prev;
} oq_halo;

/* out = D in (or D^dag) on a sub-domain: oq_dw_apply with the time hops that
 * leave the sub-domain taken from the faces (packed from the full input
 * fields by the neighbours with subset OQ_FULL).  OQ_F64 / F32 / BF16 / F16. */
int oq_dw_apply_halo(oq_handle h, int lat, int prec, const void* in_dev, void* out_dev, int nrhs, int dagger,
                     const oq_halo* halo, void* stream);

/* One pass of Dhat = D_ee - D_eo D_oo^-1 D_oe (the two passes of
 * oq_dw_hat_apply, Sec. 3 even-odd ordering):
 *   pass 1: out_o = A_oo^-1 (-1/2 H_oe in_e)          (in: even half fields)
 *   pass 2: out_e = A_ee in2_e + 1/2 H_eo in_o         (in: odd, in2: even)
 * so that Dhat in_e = pass2(pass1(in_e), in_e).  halo: the faces of the input
 * field of the pass (packed with subset OQ_EVEN for pass 1, OQ_ODD for pass
 * 2); required on a sub-domain, NULL on a whole lattice (periodic or
 * antiperiodic wrap as for oq_dw_hat_apply).  in and out must not overlap. */
int oq_dhat_pass(oq_handle h, int lat, int prec, int pass, const void* in_dev, const void* in2_dev, void* out_dev,
                 int nrhs, int dagger, const oq_halo* halo, void* stream);

/* y_k = a_host[k] x_k + b_host[k] y_k for right-hand side k < nrhs (<= 64),
 * on packed OQ_F64 or OQ_F32 fields of the subset: the vector step of a
 * solver driven from the host (the distributed CGNE over sub-domains).
 * Asynchronous. */
int oq_axpby(oq_handle h, int lat, int prec, int subset, const double* a_host, const void* x_dev,
             const double* b_host, void* y_dev, int nrhs, void* stream);

/* CGNE with reset steps (Sec. 2, Fig. 4): solves Dhat^dag Dhat psi = eta on
 * the even sites.  eta_dev / psi_dev: canonical binary64 full-lattice fields
 * (odd sites ignored on input, zero on output); psi_dev is overwritten (no
 * initial guess).  Regular steps store vectors in p->sdtype with binary32
 * arithmetic; reductions, the solution and reset-step residuals are
 * binary64.  Stops when the binary64 residual ||eta - Dhat^dag Dhat psi|| <=
 * res ||eta||, or after nmx regular steps (OQ_ERR_NOCONV).  st: host array
 * of nrhs entries.  eta_dev and psi_dev may also be page-locked host memory
 * (cudaHostAlloc or cudaHostRegister; CUDA maps it into the device's address
 * space at the same address): the solver's packing kernel then reads the
 * sources and its unpacking kernel writes the solutions over the host-device
 * link, with no separate copy.  Any other pointer (pageable host memory)
 * gives OQ_ERR_ARG. */
int oq_cgne_solve(oq_handle h, int lat, const oq_solver_params* p, const double* eta_dev,
                  double* psi_dev, int nrhs, oq_status* st, void* stream);

/* oq_cgne_solve with eta_dev / psi_dev holding the even sites only, in the
 * even-site canonical layout: nrhs consecutive fields of V/2 sites, the even
 * site with lexicographic index n (time slowest) at position n / 2, 12
 * complex binary64 per site (spin-major).  Half the bytes of the full
 * canonical fields, the same solve. */
int oq_cgne_solve_even(oq_handle h, int lat, const oq_solver_params* p, const double* eta_dev,
                       double* psi_dev, int nrhs, oq_status* st, void* stream);

/* The CGNE of oq_cgne_solve over an uneven batch: nsys systems, system k on
 * lattice lats[k] of the handle (lattices of different sizes and operators,
 * e.g. the QCD+QED charges of a U(3) ensemble), one right-hand side each
 * (eta_dev[k], psi_dev[k]: host arrays of device pointers to canonical
 * binary64 full-lattice fields).  Every stencil pass of all systems is one
 * launch of a persistent grid over a (system, site block) tile list; chunks
 * of regular iterations are captured once into a CUDA graph and replayed.
 * All systems must use the same link format.  Runs on a library-owned
 * stream after synchronising `stream`; returns when done.  st: nsys entries. */
int oq_cgne_solve_batch(oq_handle h, int nsys, const int* lats, const oq_solver_params* p,
                        const double* const* eta_dev, double* const* psi_dev, oq_status* st, void* stream);

/* Flexible GCR preconditioned by the Schwarz alternating procedure (Sec. 3,
 * 3.1, Table 2): solves D psi = eta on the full lattice.  eta_dev / psi_dev:
 * canonical binary64 full-lattice fields (nrhs consecutive, solved one after
 * the other); psi_dev is overwritten.  Each GCR step applies p->ncy Schwarz
 * cycles (all blocks of colour 0 then of colour 1, each block solved by
 * p->nmr minimal-residual steps on the block operator with Dirichlet
 * boundaries; blocks of p->bs sites, an even number per direction, at most
 * 256 sites); ncy = 0 means no preconditioner.  p->adaptive selects the
 * adaptive variant of Sec. 3.2 (ncy, nmr become maxima; MR exits after >= 4
 * steps when ||r|| > alpha ||r_prev||, when ||r|| grows, or below
 * res ||eta|| / n_blocks; cycles end when one does not lower the SAP
 * residual).  Krylov vectors, SAP and regular steps: binary32 (p->sdtype
 * must be OQ_F32); solution, restart residuals and reductions: binary64.
 * nkv (<= 64) vectors per restart, nmx GCR steps at most. */
int oq_sap_gcr_solve(oq_handle h, int lat, const oq_solver_params* p, const double* eta_dev,
                     double* psi_dev, int nrhs, oq_status* st, void* stream);

/* Learned preconditioner (not in the paper): a gauge-equivariant
 * parallel-transport network of two linear layers, 1 -> 2 -> 1 spinor
 * fields (12 -> 24 -> 12 complex channels per site),
 *   out_c'(x) = sum_q sum_c W[q][c'][c] (T_q in_c)(x),
 * over the 9 paths q = 0 (identity), 1+2mu (U_mu(x) in(x+mu)),
 * 2+2mu (U_mu(x-mu)^dag in(x-mu)) with the time-boundary factor, W a
 * complex 4x4 spin matrix.  weights_dev: binary32 master weights, 1152
 * floats = layer 1 W1[9][2][1][4][4] then layer 2 W2[9][1][2][4][4],
 * complex (re, im) interleaved; the layers use them rounded to bfloat16
 * with binary32 accumulation.  Fields: packed binary32 full fields.
 *
 * oq_nnprec_apply: out = M in.
 * oq_nnprec_grad:  gradient (binary64, 1152 doubles, d/dRe + i d/dIm of
 *   the loss) and loss = mean_k ||M r_k - e_k||^2 / ||e_k||^2 over n pairs
 *   (r_dev, e_dev: n consecutive packed binary32 full fields).
 * oq_nnprec_train: `steps` Adam steps (learning rate lr) on the mean loss,
 *   updating weights_dev in place; loss_host[step] (may be null) gets the
 *   loss before each step.  Synchronises `stream`.
 * oq_nn_gcr_solve: oq_sap_gcr_solve with M as the preconditioner of the
 *   flexible GCR instead of SAP.  SAP-GCR is the fallback: when a restart
 *   cycle (nkv steps) with the network does not halve the binary64 residual,
 *   the rest of the solve uses SAP with p->ncy, p->nmr, p->bs (no
 *   preconditioner if p->ncy = 0) and st->nn_fallback is set. */
int oq_nnprec_apply(oq_handle h, int lat, const float* weights_dev, const void* in_dev, void* out_dev,
                    void* stream);
int oq_nnprec_grad(oq_handle h, int lat, const float* weights_dev, const void* r_dev, const void* e_dev,
                   int n, double* grad_dev, double* loss_host, void* stream);
int oq_nnprec_train(oq_handle h, int lat, float* weights_dev, const void* r_dev, const void* e_dev, int n,
                    double lr, int steps, double* loss_host, void* stream);
int oq_nn_gcr_solve(oq_handle h, int lat, const oq_solver_params* p, const float* weights_dev,
                    const double* eta_dev, double* psi_dev, int nrhs, oq_status* st, void* stream);

/* oq_nnprec_apply with the channel contraction on the 5th-generation tensor
 * cores (tcgen05.mma, bfloat16 operands: weights and transported inputs,
 * binary32 accumulation in tensor memory), 128 sites per CTA.  The
 * transports stay on the CUDA cores.  Synchronises `stream`; returns
 * OQ_ERR_TIMEOUT if a bounded wait for the tensor core gave up. */
int oq_nnprec_apply_tc(oq_handle h, int lat, const float* weights_dev, const void* in_dev, void* out_dev,
                       void* stream);

/* The SAP preconditioner alone (Sec. 3): phi = M_SAP rho, starting from
 * phi = 0, p->ncy cycles of p->nmr block MR steps (blocks p->bs; p->adaptive
 * switches on the MR exit rules of Sec. 3.2 with exit-3 tolerance mr_tol; the
 * cycle test needs the global residual and is applied by oq_sap_gcr_solve
 * only).  rho_dev, phi_dev: packed binary32 full fields. */
int oq_sap_apply(oq_handle h, int lat, const oq_solver_params* p, const void* rho_dev, void* phi_dev,
                 double mr_tol, void* stream);

/* Instrumentation: while profiling is on, every stencil launch is bracketed
 * by CUDA events on its own stream, and the kernel records how many
 * right-hand sides were live in it (a solver launches its regular steps in
 * chunks and gates off, on the device, every right-hand side whose state has
 * left the step's mode).  oq_profile_stop() synchronises the device and
 * returns one entry per (mode, epilogue, precision, rhs per thread, link
 * format, adjoint): mode 0 = full Dw, 1 = Dhat pass 1 (odd sites), 2 = Dhat
 * pass 2 (even sites); epi 0 = plain store, 1 = store + norm, 2 = fused CG
 * update, 3 = reset residual; link_fmt -1 for binary64 / double-float links.
 * launches, total_ms and bytes cover the launches with at least one live
 * right-hand side: bytes = algorithmic bytes (each operand counted once:
 * links and clover once per launch, spinor and epilogue vectors per live
 * right-hand side); rhs_launches = the sum of live right-hand sides over
 * those launches.  Launches with no live right-hand side move no operand:
 * they are counted in gated_launches / gated_ms only.  The first 262,144
 * launches of a profile are recorded this way, later ones count as fully
 * live. */
typedef struct {
  int mode, epi, prec, launches;
  double total_ms;
  double bytes;
  int nr, link_fmt;
  int dag;  /* 1: the adjoint (Dhat^dag / Dw^dag) instantiation */
  int gated_launches;
  double gated_ms;
  long long rhs_launches;
} oq_kernel_time;
int oq_profile_start(oq_handle h);
/* Number of kernels the library has launched through this handle so far. */
long long oq_kernel_launches(oq_handle h);
int oq_profile_stop(oq_handle h, oq_kernel_time* out, int max_entries, int* n_entries);

#ifdef __cplusplus
}
#endif

#endif /* OQ_H */
