// Tensor-core (tcgen05) form of the PTC layer's channel contraction.
//
// For every (site, colour a) row the layer is a dense product
//   Y[row][n] = sum_k X[row][k] W[n][k],   k = (path q, c_in, spin t),
//                                          n = (c_out, spin s),
// complex; written as a real product with X' = [Re X | Im X] and
// W' = [[Re W, -Im W], [Im W, Re W]] (rows n' = (re|im, n)), both in bfloat16,
// accumulated in binary32 in tensor memory:
//   D (128 x N') = X' (128 x K') . W'^T,   M = 128, N' = 16, K' padded to 16.
// One CTA = 42 sites = 126 rows (row = 3 site + colour; rows 126, 127 zero),
// 4 warps.  The gather (transport of every input along every path, binary32
// CUDA-core work) is split into (site, path) items over all threads, which
// write their entries of X' into shared memory in the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per core matrix; LBO = next core
// along K, SBO = next 8-row group).  One elected thread issues the
// tcgen05.mma instructions, commits them to an mbarrier, every thread waits
// (bounded), then reads its row of the accumulator with tcgen05.ld (warp w
// owns TMEM lanes 32w..32w+31) and stores its colour of the output spinors.
#include <math.h>
#include <stdint.h>

#include "../../include/oq.h"
#include "ctx.h"
#include "oq_kernels.h"

namespace oq {

static const int TC_M = 128;
static const int TC_N = 16;        // N' (real-embedded outputs, padded)
static const int TC_COLS = 32;     // TMEM columns allocated (one 128 x 16 accumulator)
static const int TC_SITES = 42;    // sites per CTA: rows 3 * site + colour, 126 of 128 used
static const unsigned TC_SPIN_LIMIT = 1u << 26;

struct PtcTcArgs {
  Geom g;
  const void* links;
  const char* in;
  char* out;
  long fbytes, hbytes;
  const float2* w;  // binary32 master weights of this layer [9][COUT][CIN][4][4]
  int* error;       // set to 1 if a bounded wait gave up
  unsigned long long wait_ns;  // limit of the wait for the tensor core
  int skip_commit;  // test hook: issue no MMA, so that the bounded wait runs out
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// no-swizzle K-major shared-memory matrix descriptor (tcgen05)
__device__ __forceinline__ uint64_t make_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
  return d;              // base offset 0, absolute-LBO mode off, layout type 0 (no swizzle)
}

// instruction descriptor: kind::f16, A = B = bf16, D = f32, both K-major
__host__ __device__ constexpr uint32_t make_idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// byte offset of element (row, k) in a no-swizzle K-major tile with kp columns
__device__ __forceinline__ uint32_t core_off(int row, int k, int kp) {
  return (uint32_t)(((row >> 3) * (kp >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ __nv_bfloat16 bf(float v) { return __float2bfloat16_rn(v); }

template <int FMT>
__device__ __forceinline__ void tc_transport(const PtcTcArgs& a, const char* f, int q, int p, long i, const int x[4],
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

// W' (bfloat16, core-matrix layout) from the binary32 master weights, once per call
template <int CIN, int COUT>
__global__ void ptc_tc_prepare_b(const float2* __restrict__ w, unsigned char* __restrict__ bglob) {
  constexpr int K = 9 * CIN * 4;
  constexpr int KP = ((2 * K + 15) / 16) * 16;
  constexpr int N = COUT * 4;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < TC_N * KP; e += gridDim.x * blockDim.x) {
    const int n2 = e / KP, k2 = e % KP;
    float v = 0.f;
    if (n2 < 2 * N && k2 < 2 * K) {
      const int n = n2 % N, im_row = n2 / N;
      const int k = k2 % K, im_col = k2 / K;
      const int co = n / 4, s = n % 4;
      const int q = k / (CIN * 4), ci = (k / 4) % CIN, t = k % 4;
      const float2 wv = w[((q * COUT + co) * CIN + ci) * 16 + s * 4 + t];
      v = im_row == 0 ? (im_col == 0 ? wv.x : -wv.y) : (im_col == 0 ? wv.y : wv.x);
    }
    *reinterpret_cast<__nv_bfloat16*>(bglob + core_off(n2, k2, KP)) = bf(v);
  }
}

// Persistent over 42-site tiles: TMEM, the mbarrier and W' in shared memory
// are set up once per CTA; per tile: gather -> MMA -> bounded wait -> read
// the accumulator -> store.  The mbarrier phase flips every tile.
template <int FMT, int CIN, int COUT>
__global__ void __launch_bounds__(128) ptc_tc_kernel(const PtcTcArgs a, const uint4* __restrict__ bglob) {
  constexpr int K = 9 * CIN * 4;                // complex inputs of one (site, colour) row
  constexpr int KP = ((2 * K + 15) / 16) * 16;  // real-embedded, padded to the MMA K step
  constexpr int N = COUT * 4;                   // complex outputs
  constexpr uint32_t A_BYTES = TC_M * KP * 2;
  constexpr uint32_t B_BYTES = TC_N * KP * 2;
  extern __shared__ __align__(1024) unsigned char sm[];
  // layout: [A | B | mbarrier | tmem slot]
  unsigned char* A = sm;
  unsigned char* B = sm + A_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + A_BYTES + B_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "n"(TC_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int e = tid; e < (int)(B_BYTES / 16); e += blockDim.x) reinterpret_cast<uint4*>(B)[e] = bglob[e];
  // constant zeros of A': the K padding of every row, and rows 126, 127
  for (int e = tid; e < TC_M * (KP - 2 * K); e += blockDim.x) {
    const int r = e / (KP - 2 * K), k = 2 * K + e % (KP - 2 * K);
    *reinterpret_cast<__nv_bfloat16*>(A + core_off(r, k, KP)) = bf(0.f);
  }
  for (int e = tid; e < (TC_M - 3 * TC_SITES) * 2 * K; e += blockDim.x) {
    const int r = 3 * TC_SITES + e / (2 * K), k = e % (2 * K);
    *reinterpret_cast<__nv_bfloat16*>(A + core_off(r, k, KP)) = bf(0.f);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const long ntile = (2 * a.g.Vh + TC_SITES - 1) / TC_SITES;
  uint32_t phase = 0;

  for (long tile = blockIdx.x; tile < ntile; tile += gridDim.x) {
    const long site0 = tile * TC_SITES;
    // A': row 3 * (site in tile) + colour; (site, path) items over all threads
    // items run fastest over sites, so that a warp gathers neighbouring sites
    // (coalesced loads) and writes rows 48 bytes apart (few bank conflicts)
    for (int item = tid; item < TC_SITES * 9; item += blockDim.x) {
      const int ls = item % TC_SITES, q = item / TC_SITES;
      const long j = site0 + ls;
      const bool live = j < 2 * a.g.Vh;
      const int p = (live && j >= a.g.Vh) ? 1 : 0;
      const long i = live ? j - p * a.g.Vh : 0;
      int x[4];
      eo_coords(a.g, p, i, x);
#pragma unroll
      for (int ci = 0; ci < CIN; ++ci) {
        Spinor<float> t;
        if (live)
          tc_transport<FMT>(a, a.in + ci * a.fbytes, q, p, i, x, t);
        else
#pragma unroll
          for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int c = 0; c < 3; ++c) t.c[s][c] = cx<float>{0.f, 0.f};
        // spins (s, s+1) are adjacent columns of one core matrix: 4-byte stores
#pragma unroll
        for (int s = 0; s < 4; s += 2) {
          const int k = (q * CIN + ci) * 4 + s;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            const int row = 3 * ls + c;
            *reinterpret_cast<__nv_bfloat162*>(A + core_off(row, k, KP)) =
                __floats2bfloat162_rn(t.c[s][c].re, t.c[s + 1][c].re);
            *reinterpret_cast<__nv_bfloat162*>(A + core_off(row, K + k, KP)) =
                __floats2bfloat162_rn(t.c[s][c].im, t.c[s + 1][c].im);
          }
        }
      }
    }
    // make the generic-proxy smem writes visible to the tensor core (async proxy)
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

    if (tid == 0 && !a.skip_commit) {
      constexpr uint32_t idesc = make_idesc(TC_M, TC_N);
      constexpr uint32_t SBO = (KP / 8) * 128;
      const uint32_t a_base = smem_u32(A);
      const uint32_t b_base = smem_u32(B);
#pragma unroll
      for (int ks = 0; ks < KP / 16; ++ks) {
        const uint64_t ad = make_desc(a_base + ks * 256, 128, SBO);
        const uint64_t bd = make_desc(b_base + ks * 256, 128, SBO);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar)));
    }
    // bounded wait for the MMAs of this tile: give up after wait_ns of the
    // global timer (or TC_SPIN_LIMIT polls); the decision is made uniform over
    // the CTA, which then flags the error, skips the remaining tiles and frees TMEM
    uint32_t done = 0;
    {
      unsigned n = 0;
      uint64_t t0, t1;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      while (!done && n < TC_SPIN_LIMIT) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(mbar)), "r"(phase));
        ++n;
        if (!done) {
          asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
          if (t1 - t0 > a.wait_ns) break;
        }
      }
    }
    if (__syncthreads_or(done ? 0 : 1)) {
      if (tid == 0 && a.error) atomicExch(a.error, 1);
      break;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // row r = tid of the accumulator: site r / 3, colour r % 3
    uint32_t rr[16];
    {
      const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(rr[0]), "=r"(rr[1]), "=r"(rr[2]), "=r"(rr[3]), "=r"(rr[4]), "=r"(rr[5]), "=r"(rr[6]),
            "=r"(rr[7]), "=r"(rr[8]), "=r"(rr[9]), "=r"(rr[10]), "=r"(rr[11]), "=r"(rr[12]), "=r"(rr[13]),
            "=r"(rr[14]), "=r"(rr[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    }
    if (tid < 3 * TC_SITES) {
      const int ls = tid / 3, c = tid % 3;
      const long j = site0 + ls;
      if (j < 2 * a.g.Vh) {
        const int p = j >= a.g.Vh ? 1 : 0;
        const long i = j - p * a.g.Vh;
#pragma unroll
        for (int co = 0; co < COUT; ++co) {
          float2* base = reinterpret_cast<float2*>(a.out + co * a.fbytes + (long)p * a.hbytes);
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            const int k = s * 3 + c;  // complex component of the site vector
            base[((long)(k >> 1) * a.g.Vh + i) * 2 + (k & 1)] =
                make_float2(__uint_as_float(rr[co * 4 + s]), __uint_as_float(rr[N + co * 4 + s]));
          }
        }
      }
    }
    // every thread has read the accumulator before the next tile's MMA writes it
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TC_COLS));
  }
}

template <int CIN, int COUT>
static cudaError_t ptc_tc_layer(const PtcTcArgs& a, int fmt, unsigned char* bglob, int nsm, cudaStream_t s) {
  constexpr int K = 9 * CIN * 4;
  constexpr int KP = ((2 * K + 15) / 16) * 16;
  const size_t smem = (size_t)TC_M * KP * 2 + (size_t)TC_N * KP * 2 + 16;
  ptc_tc_prepare_b<CIN, COUT><<<8, 256, 0, s>>>(a.w, bglob);
  const long ntile = (2 * a.g.Vh + TC_SITES - 1) / TC_SITES;
  const long cap = (long)nsm * 8;
  dim3 grid((unsigned)(ntile < cap ? ntile : cap)), block(128);
  const uint4* b = reinterpret_cast<const uint4*>(bglob);
  if (fmt == LINK_12) {
    cudaFuncSetAttribute(ptc_tc_kernel<LINK_12, CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ptc_tc_kernel<LINK_12, CIN, COUT><<<grid, block, smem, s>>>(a, b);
  } else {
    cudaFuncSetAttribute(ptc_tc_kernel<LINK_18, CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ptc_tc_kernel<LINK_18, CIN, COUT><<<grid, block, smem, s>>>(a, b);
  }
  return cudaGetLastError();
}

}  // namespace oq

using namespace oq;

// y = L2 L1 r with the tensor-core layers (binary32 master weights, rounded
// to bfloat16 inside the kernel).  Returns OQ_ERR_TIMEOUT if a bounded wait
// for the tensor core gave up.
extern "C" int oq_nnprec_apply_tc(oq_handle h, int lat, const float* weights_dev, const void* in_dev, void* out_dev,
                                  void* stream) {
  if (!h || lat < 0 || lat >= (int)h->lats.size() || !weights_dev || !in_dev || !out_dev) return OQ_ERR_ARG;
  if (!h->lats[lat].has_gauge || h->lats[lat].halo_t) return OQ_ERR_STATE;  // whole lattices only
  return nnprec_forward_tc(h, lat, weights_dev, in_dev, out_dev, (cudaStream_t)stream);
}

int oq::nnprec_forward_tc(oq_handle h, int lat, const float* weights_dev, const void* in_dev, void* out_dev,
                          cudaStream_t s) {
  LatCtx& L = h->lats[lat];
  const long hb = spinor_half_bytes(L.g.Vh, P_F32);
  void *hid, *bglob;
  int rc = h->workspace(lat, "nntc_hid", 2 * 2 * hb, &hid);
  if (!rc) rc = h->workspace(lat, "nntc_b", 16 * 160 * 2 + 16 * 144 * 2, &bglob);
  if (!rc) rc = h->ensure_scratch();
  if (rc) return rc;
  int nsm = 152;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, h->device);
  unsigned char* b1 = (unsigned char*)bglob;          // layer 1: 16 x 80 bf16
  unsigned char* b2 = b1 + 16 * 80 * 2;               // layer 2: 16 x 144 bf16 (16-byte aligned)
  if (cudaMemsetAsync(h->status_dev, 0, sizeof(int), s) != cudaSuccess) return OQ_ERR_CUDA;
  PtcTcArgs a;
  a.g = L.g;
  a.links = L.u32.p;
  a.hbytes = hb;
  a.fbytes = 2 * hb;
  a.error = h->status_dev;
  a.wait_ns = 1000000000ull;  // 1 s
  a.skip_commit = h->hook_tc_skip_commit ? 1 : 0;
  a.in = (const char*)in_dev;
  a.out = (char*)hid;
  a.w = (const float2*)weights_dev;
  if (ptc_tc_layer<1, 2>(a, L.link_fmt, b1, nsm, s) != cudaSuccess) return OQ_ERR_CUDA;
  a.in = (const char*)hid;
  a.out = (char*)out_dev;
  a.w = (const float2*)weights_dev + 9 * 2 * 1 * 16;
  if (ptc_tc_layer<2, 1>(a, L.link_fmt, b2, nsm, s) != cudaSuccess) return OQ_ERR_CUDA;
  h->launches += 4;
  int err = 0;
  if (cudaMemcpyAsync(&err, h->status_dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return OQ_ERR_CUDA;
  return err ? OQ_ERR_TIMEOUT : OQ_OK;
}
