// Tensor-core (tcgen05) form of the PTC layer's channel contraction.
//
// For a tile of 128 sites and one colour a, the layer is a dense product
//   Y_a[site][n] = sum_k X_a[site][k] W[n][k],   k = (path q, c_in, spin t),
//                                                 n = (c_out, spin s),
// complex; written as a real product with X' = [Re X | Im X] and
// W' = [[Re W, -Im W], [Im W, Re W]] (rows n' = (re|im, n)), both in bfloat16,
// accumulated in binary32 in tensor memory:
//   D_a (128 x N') = X'_a (128 x K') . W'^T,   M = 128, N' = 16, K' padded to 16.
// One CTA = 128 sites = 4 warps; every thread gathers and transports the
// inputs of its own site (binary32 CUDA-core work) and writes row `site` of
// the three operand tiles X'_a into shared memory in the no-swizzle K-major
// core-matrix layout (8 rows x 16 bytes per core matrix; LBO = next core
// along K, SBO = next 8-row group).  One elected thread issues the
// tcgen05.mma instructions for the 3 colours, commits them to an mbarrier,
// every thread waits (bounded), then reads its row of the accumulators with
// tcgen05.ld (warp w owns TMEM lanes 32w..32w+31) and stores the outputs.
#include <math.h>
#include <stdint.h>

#include "../../include/oq.h"
#include "ctx.h"
#include "oq_kernels.h"

namespace oq {

static const int TC_M = 128;
static const int TC_N = 16;        // N' (real-embedded outputs, padded)
static const int TC_COLS = 128;    // TMEM columns allocated (accumulators at 0, 32, 64)
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
  const long j = eo_neighbour(a.g, x, mu, fwd ? +1 : -1, &cr);
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
__global__ void __launch_bounds__(128) ptc_tc_kernel(const PtcTcArgs a) {
  constexpr int K = 9 * CIN * 4;             // complex inputs per colour row
  constexpr int KP = ((2 * K + 15) / 16) * 16;  // real-embedded, padded to the MMA K step
  constexpr int N = COUT * 4;                // complex outputs
  constexpr uint32_t A_BYTES = TC_M * KP * 2;
  constexpr uint32_t B_BYTES = TC_N * KP * 2;
  extern __shared__ __align__(1024) unsigned char sm[];
  // layout: [A_0 | A_1 | A_2 | B | pad (one A tile) | mbarrier | tmem slot]
  unsigned char* A = sm;
  unsigned char* B = sm + 3 * A_BYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + 4 * A_BYTES + B_BYTES);
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
  // B' = [[Re W, -Im W], [Im W, Re W]] rows n' = re/im x (c_out, s); zero padded
  for (int e = tid; e < TC_N * KP; e += blockDim.x) {
    const int n2 = e / KP, k2 = e % KP;
    float v = 0.f;
    if (n2 < 2 * N && k2 < 2 * K) {
      const int n = n2 % N, im_row = n2 / N;
      const int k = k2 % K, im_col = k2 / K;
      const int co = n / 4, s = n % 4;
      const int q = k / (CIN * 4), ci = (k / 4) % CIN, t = k % 4;
      const float2 w = a.w[((q * COUT + co) * CIN + ci) * 16 + s * 4 + t];
      v = im_row == 0 ? (im_col == 0 ? w.x : -w.y) : (im_col == 0 ? w.y : w.x);
    }
    *reinterpret_cast<__nv_bfloat16*>(B + core_off(n2, k2, KP)) = bf(v);
  }
  // A'_a rows: this thread's site, all paths and input channels
  const long j = (long)blockIdx.x * TC_M + tid;
  const bool live = j < 2 * a.g.Vh;
  const int p = (live && j >= a.g.Vh) ? 1 : 0;
  const long i = live ? j - p * a.g.Vh : 0;
  int x[4];
  eo_coords(a.g, p, i, x);
  for (int q = 0; q < 9; ++q) {
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
#pragma unroll
      for (int s = 0; s < 4; ++s) {
        const int k = (q * CIN + ci) * 4 + s;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          unsigned char* Ac = A + c * A_BYTES;
          *reinterpret_cast<__nv_bfloat16*>(Ac + core_off(tid, k, KP)) = bf(t.c[s][c].re);
          *reinterpret_cast<__nv_bfloat16*>(Ac + core_off(tid, K + k, KP)) = bf(t.c[s][c].im);
        }
      }
    }
  }
  for (int k = 2 * K; k < KP; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) *reinterpret_cast<__nv_bfloat16*>(A + c * A_BYTES + core_off(tid, k, KP)) = bf(0.f);
  // make the generic-proxy smem writes visible to the tensor core (async proxy)
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  if (tid == 0 && !a.skip_commit) {
    constexpr uint32_t idesc = make_idesc(TC_M, TC_N);
    constexpr uint32_t SBO = (KP / 8) * 128;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const uint32_t a_base = smem_u32(A + c * A_BYTES);
      const uint32_t b_base = smem_u32(B);
#pragma unroll
      for (int ks = 0; ks < KP / 16; ++ks) {
        const uint64_t ad = make_desc(a_base + ks * 256, 128, SBO);
        const uint64_t bd = make_desc(b_base + ks * 256, 128, SBO);
        const uint32_t d_tmem = tmem + (uint32_t)(32 * c);
        const uint32_t acc = ks > 0 ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
      }
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
        smem_u32(mbar)));
  }
  // bounded wait for the MMAs (phase 0): give up after wait_ns of the global
  // timer (or TC_SPIN_LIMIT polls), flag the error and carry on to free TMEM
  {
    uint32_t done = 0;
    unsigned n = 0;
    uint64_t t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    while (!done && n < TC_SPIN_LIMIT) {
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(smem_u32(mbar)), "r"(0u));
      ++n;
      if (!done) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        if (t1 - t0 > a.wait_ns) break;
      }
    }
    if (!done && a.error) atomicExch(a.error, 1);
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  // read row `tid` of the three accumulators
  float d[3][16];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(32 * c);
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int k = 0; k < 16; ++k) d[c][k] = __uint_as_float(r[k]);
  }
  if (live) {
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
      Spinor<float> o;
#pragma unroll
      for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int c = 0; c < 3; ++c) o.c[s][c] = cx<float>{d[c][co * 4 + s], d[c][N + co * 4 + s]};
      store_spinor<P_F32>(a.out + co * a.fbytes + (long)p * a.hbytes, a.g.Vh, i, o);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TC_COLS));
  }
}

template <int CIN, int COUT>
static cudaError_t ptc_tc_layer(const PtcTcArgs& a, int fmt, cudaStream_t s) {
  constexpr int K = 9 * CIN * 4;
  constexpr int KP = ((2 * K + 15) / 16) * 16;
  const size_t smem = 4 * (size_t)TC_M * KP * 2 + (size_t)TC_N * KP * 2 + 16;
  dim3 grid((unsigned)((2 * a.g.Vh + TC_M - 1) / TC_M)), block(128);
  if (fmt == LINK_12) {
    cudaFuncSetAttribute(ptc_tc_kernel<LINK_12, CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ptc_tc_kernel<LINK_12, CIN, COUT><<<grid, block, smem, s>>>(a);
  } else {
    cudaFuncSetAttribute(ptc_tc_kernel<LINK_18, CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    ptc_tc_kernel<LINK_18, CIN, COUT><<<grid, block, smem, s>>>(a);
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
  LatCtx& L = h->lats[lat];
  if (!L.has_gauge) return OQ_ERR_STATE;
  cudaStream_t s = (cudaStream_t)stream;
  const long hb = spinor_half_bytes(L.g.Vh, P_F32);
  void* hid;
  int rc = h->workspace(lat, "nntc_hid", 2 * 2 * hb, &hid);
  if (!rc) rc = h->ensure_scratch();
  if (rc) return rc;
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
  if (ptc_tc_layer<1, 2>(a, L.link_fmt, s) != cudaSuccess) return OQ_ERR_CUDA;
  a.in = (const char*)hid;
  a.out = (char*)out_dev;
  a.w = (const float2*)weights_dev + 9 * 2 * 1 * 16;
  if (ptc_tc_layer<2, 1>(a, L.link_fmt, s) != cudaSuccess) return OQ_ERR_CUDA;
  h->launches += 2;
  int err = 0;
  if (cudaMemcpyAsync(&err, h->status_dev, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return OQ_ERR_CUDA;
  return err ? OQ_ERR_TIMEOUT : OQ_OK;
}
