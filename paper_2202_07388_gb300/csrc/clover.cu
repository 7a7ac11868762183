// Clover term: A(x) = (4 + m0) + c_sw (i/4) sum_{mu,nu} sigma_{mu nu} F_{mu nu}(x)
// (QCD+QED with separate coefficients: c_sw F -> c_sw F^{SU(3)} + c_sw^QED
// F^{U(1)} 1_colour; Schroedinger-functional lattices: 4 + m0 + c_F - 1 at
// x0 = 1 and T-1)
// with the clover-leaf field strength F = (Q - Q^dag)/8, Q the sum of the four
// plaquettes at x in the (mu, nu) plane.  In the chiral basis
// sigma_{0k} = diag(s_k, -s_k) and sigma_{jk} = -eps_{jkl} diag(s_l, s_l), so A
// splits into two Hermitian 6x6 blocks (index 3*spin + colour):
//
//   block(+) = c0 + sum_k s_k (x) (i c_sw / 2)(F_0k - Fd_k)
//   block(-) = c0 - sum_k s_k (x) (i c_sw / 2)(F_0k + Fd_k)
//
// with Fd_1 = F_23, Fd_2 = -F_13, Fd_3 = F_12 and c0 = 4 + m0.  Everything
// is built and inverted in binary64 (Gauss-Jordan with partial pivoting),
// then stored in binary64 and binary32.  One thread per site.
#include "oq_internal.h"
#include "oq_kernels.h"

namespace oq {

typedef cx<double> cd;
struct M3 {
  cd m[3][3];
};

__device__ __forceinline__ M3 mul(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cd s = a.m[i][0] * b.m[0][j];
      cfma(s, a.m[i][1], b.m[1][j]);
      cfma(s, a.m[i][2], b.m[2][j]);
      c.m[i][j] = s;
    }
  return c;
}
// a * b^dag
__device__ __forceinline__ M3 mul_d(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cd s = a.m[i][0] * conj(b.m[j][0]);
      cfma(s, a.m[i][1], conj(b.m[j][1]));
      cfma(s, a.m[i][2], conj(b.m[j][2]));
      c.m[i][j] = s;
    }
  return c;
}
// a^dag * b
__device__ __forceinline__ M3 dmul(const M3& a, const M3& b) {
  M3 c;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      cd s = cmulc(a.m[0][i], b.m[0][j]);
      cfmac(s, a.m[1][i], b.m[1][j]);
      cfmac(s, a.m[2][i], b.m[2][j]);
      c.m[i][j] = s;
    }
  return c;
}

// y += d mu (d = -1, 0, +1) on the periodic lattice, with the x1 shift of a
// C* boundary when the step wraps
__device__ __forceinline__ void displace(const Geom& g, int y[4], int mu, int d) {
  if (!d) return;
  int v = y[mu] + d;
  const bool wrap = v < 0 || v >= g.L[mu];
  y[mu] = (v + g.L[mu]) % g.L[mu];
  if (wrap) y[1] = cs_x1(g, mu, y[1]);
}

// the link U_mu(y), y = x + d1 mu1 + d2 mu2; with au1 times exp(i q A_mu(y))
__device__ __forceinline__ M3 link_at(const Geom& g, const double2* u64, const int x[4], int mu, int d1, int mu1,
                                      int d2, int mu2, const double* au1 = nullptr, double q = 0.0) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  displace(g, y, mu1, d1);
  displace(g, y, mu2, d2);
  const int p = (y[0] + y[1] + y[2] + y[3]) & 1;
  const long j = eo_index(g, y);
  Su3<double> u;
  load_link<double, LINK_18>(u64, g.Vh, p, mu, j, u);
  cd ph = cd{1.0, 0.0};
  if (au1) {
    double sn, cs;
    sincos(q * au1[(long)(p * 4 + mu) * g.Vh + j], &sn, &cs);
    ph = cd{cs, sn};
  }
  M3 r;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) r.m[a][b] = au1 ? u.m[a][b] * ph : u.m[a][b];
  return r;
}

// F_{mu nu}(x) = (Q - Q^dag) / 8 (au1: of the links times exp(i q A))
__device__ M3 field_strength(const Geom& g, const double2* u64, const int x[4], int mu, int nu,
                             const double* au1 = nullptr, double qc = 0.0) {
  M3 umx = link_at(g, u64, x, mu, 0, 0, 0, 0, au1, qc);
  M3 unx = link_at(g, u64, x, nu, 0, 0, 0, 0, au1, qc);
  M3 un_xpm = link_at(g, u64, x, nu, +1, mu, 0, 0, au1, qc);
  M3 um_xpn = link_at(g, u64, x, mu, +1, nu, 0, 0, au1, qc);
  M3 um_xmm = link_at(g, u64, x, mu, -1, mu, 0, 0, au1, qc);
  M3 un_xmm = link_at(g, u64, x, nu, -1, mu, 0, 0, au1, qc);
  M3 um_xmm_pn = link_at(g, u64, x, mu, -1, mu, +1, nu, au1, qc);
  M3 um_xmn = link_at(g, u64, x, mu, -1, nu, 0, 0, au1, qc);
  M3 un_xmn = link_at(g, u64, x, nu, -1, nu, 0, 0, au1, qc);
  M3 um_xmm_mn = link_at(g, u64, x, mu, -1, mu, -1, nu, au1, qc);
  M3 un_xmm_mn = link_at(g, u64, x, nu, -1, mu, -1, nu, au1, qc);
  M3 un_xpm_mn = link_at(g, u64, x, nu, +1, mu, -1, nu, au1, qc);
  // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^dag U_nu(x)^dag
  M3 q = mul_d(mul_d(mul(umx, un_xpm), um_xpn), unx);
  // leaf 2: U_nu(x) U_mu(x-mu+nu)^dag U_nu(x-mu)^dag U_mu(x-mu)
  M3 l2 = mul(mul_d(mul_d(unx, um_xmm_pn), un_xmm), um_xmm);
  // leaf 3: U_mu(x-mu)^dag U_nu(x-mu-nu)^dag U_mu(x-mu-nu) U_nu(x-nu)
  M3 l3 = mul(dmul(um_xmm, dmul(un_xmm_mn, um_xmm_mn)), un_xmn);
  // leaf 4: U_nu(x-nu)^dag U_mu(x-nu) U_nu(x+mu-nu) U_mu(x)^dag
  M3 l4 = mul_d(mul(dmul(un_xmn, um_xmn), un_xpm_mn), umx);
  M3 f;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) q.m[a][b] = q.m[a][b] + l2.m[a][b] + l3.m[a][b] + l4.m[a][b];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) f.m[a][b] = 0.125 * (q.m[a][b] - conj(q.m[b][a]));
  return f;
}

// U(1) angle A_mu(y) at y = x + d1 mu1 + d2 mu2 (packed [parity][mu][site])
__device__ __forceinline__ double angle_at(const Geom& g, const double* au1, const int x[4], int mu, int d1,
                                           int mu1, int d2, int mu2) {
  int y[4] = {x[0], x[1], x[2], x[3]};
  displace(g, y, mu1, d1);
  displace(g, y, mu2, d2);
  const int p = (y[0] + y[1] + y[2] + y[3]) & 1;
  return au1[(long)(p * 4 + mu) * g.Vh + eo_index(g, y)];
}

// U(1) clover-leaf field strength of the charged links exp(i q A):
// F = (Q - Q^*) / 8 = (i/4) sum over the four leaves of sin(q theta_leaf),
// theta_leaf the oriented sum of the angles around the leaf (the same four
// leaves as field_strength); returns f with F = i f
__device__ double u1_field_strength(const Geom& g, const double* au1, double q, const int x[4], int mu, int nu) {
  const double t1 = angle_at(g, au1, x, mu, 0, 0, 0, 0) + angle_at(g, au1, x, nu, +1, mu, 0, 0) -
                    angle_at(g, au1, x, mu, +1, nu, 0, 0) - angle_at(g, au1, x, nu, 0, 0, 0, 0);
  const double t2 = angle_at(g, au1, x, nu, 0, 0, 0, 0) - angle_at(g, au1, x, mu, -1, mu, +1, nu) -
                    angle_at(g, au1, x, nu, -1, mu, 0, 0) + angle_at(g, au1, x, mu, -1, mu, 0, 0);
  const double t3 = -angle_at(g, au1, x, mu, -1, mu, 0, 0) - angle_at(g, au1, x, nu, -1, mu, -1, nu) +
                    angle_at(g, au1, x, mu, -1, mu, -1, nu) + angle_at(g, au1, x, nu, -1, nu, 0, 0);
  const double t4 = -angle_at(g, au1, x, nu, -1, nu, 0, 0) + angle_at(g, au1, x, mu, -1, nu, 0, 0) +
                    angle_at(g, au1, x, nu, +1, mu, -1, nu) - angle_at(g, au1, x, mu, 0, 0, 0, 0);
  return 0.25 * (sin(q * t1) + sin(q * t2) + sin(q * t3) + sin(q * t4));
}

// invert a general 6x6 complex matrix in place (Gauss-Jordan, partial pivoting)
__device__ bool invert6(cd a[6][6], cd inv[6][6]) {
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int j = 0; j < 6; ++j) inv[i][j] = cd{i == j ? 1.0 : 0.0, 0.0};
  for (int c = 0; c < 6; ++c) {
    int piv = c;
    double best = a[c][c].re * a[c][c].re + a[c][c].im * a[c][c].im;
    for (int r = c + 1; r < 6; ++r) {
      double v = a[r][c].re * a[r][c].re + a[r][c].im * a[r][c].im;
      if (v > best) { best = v; piv = r; }
    }
    if (!(best > 0.0)) return false;
    if (piv != c) {
      for (int j = 0; j < 6; ++j) {
        cd t = a[c][j]; a[c][j] = a[piv][j]; a[piv][j] = t;
        t = inv[c][j]; inv[c][j] = inv[piv][j]; inv[piv][j] = t;
      }
    }
    cd d = a[c][c];
    double n2 = d.re * d.re + d.im * d.im;
    cd dinv = cd{d.re / n2, -d.im / n2};
    for (int j = 0; j < 6; ++j) {
      a[c][j] = a[c][j] * dinv;
      inv[c][j] = inv[c][j] * dinv;
    }
    for (int r = 0; r < 6; ++r) {
      if (r == c) continue;
      cd f = a[r][c];
      for (int j = 0; j < 6; ++j) {
        a[r][j] = a[r][j] - f * a[c][j];
        inv[r][j] = inv[r][j] - f * inv[c][j];
      }
    }
  }
  return true;
}

// store one Hermitian block (upper triangle) into the packed arrays
__device__ __forceinline__ void store_block(const Geom& g, int p, long i, int b, const cd m[6][6],
                                            double2* a64, float4* a32) {
  double r[36];
#pragma unroll
  for (int k = 0; k < 6; ++k) r[k] = m[k][k].re;
  int k = 0;
#pragma unroll
  for (int r0 = 0; r0 < 6; ++r0)
#pragma unroll
    for (int c0 = r0 + 1; c0 < 6; ++c0) {
      // Hermitian part of the computed entry (exact for A, rounding-level for A^-1)
      r[6 + 2 * k] = 0.5 * (m[r0][c0].re + m[c0][r0].re);
      r[7 + 2 * k] = 0.5 * (m[r0][c0].im - m[c0][r0].im);
      ++k;
    }
  double2* q64 = a64 + (long)p * 36 * g.Vh;
#pragma unroll
  for (int c = 0; c < 18; ++c) q64[(18 * b + c) * g.Vh + i] = make_double2(r[2 * c], r[2 * c + 1]);
  float4* q32 = a32 + (long)p * 18 * g.Vh;
#pragma unroll
  for (int c = 0; c < 9; ++c)
    q32[(9 * b + c) * g.Vh + i] =
        make_float4((float)r[4 * c], (float)r[4 * c + 1], (float)r[4 * c + 2], (float)r[4 * c + 3]);
}

// qed: 0 = F of the links alone; 1 = F of the links times exp(i q A) (the
// U(3) clover); 2 = csw F(links) + csw_qed F(exp(i q A)) 1_colour
__global__ void __launch_bounds__(128) clover_kernel(Geom g, const double2* __restrict__ u64,
                                                     const double* __restrict__ au1, double q, int qed, double c0,
                                                     double csw, double csw_qed, double cF, double2* a64,
                                                     float4* a32, double2* i64, float4* i32, int* status) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int p = blockIdx.y;
  if (i >= g.Vh) return;
  int x[4];
  eo_coords(g, p, i, x);
  const double* ph = qed == 1 ? au1 : nullptr;
  M3 f01 = field_strength(g, u64, x, 0, 1, ph, q);
  M3 f02 = field_strength(g, u64, x, 0, 2, ph, q);
  M3 f03 = field_strength(g, u64, x, 0, 3, ph, q);
  M3 f12 = field_strength(g, u64, x, 1, 2, ph, q);
  M3 f13 = field_strength(g, u64, x, 1, 3, ph, q);
  M3 f23 = field_strength(g, u64, x, 2, 3, ph, q);
  // scale by c_sw here, so that a separate U(1) term adds with its own coefficient
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      f01.m[a][c] = csw * f01.m[a][c]; f02.m[a][c] = csw * f02.m[a][c]; f03.m[a][c] = csw * f03.m[a][c];
      f12.m[a][c] = csw * f12.m[a][c]; f13.m[a][c] = csw * f13.m[a][c]; f23.m[a][c] = csw * f23.m[a][c];
    }
  if (qed == 2) {
    // U(1) field strength i f (x) 1_colour, weighted by c_sw^QED
    const double e01 = csw_qed * u1_field_strength(g, au1, q, x, 0, 1);
    const double e02 = csw_qed * u1_field_strength(g, au1, q, x, 0, 2);
    const double e03 = csw_qed * u1_field_strength(g, au1, q, x, 0, 3);
    const double e12 = csw_qed * u1_field_strength(g, au1, q, x, 1, 2);
    const double e13 = csw_qed * u1_field_strength(g, au1, q, x, 1, 3);
    const double e23 = csw_qed * u1_field_strength(g, au1, q, x, 2, 3);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      f01.m[a][a] = f01.m[a][a] + cd{0.0, e01}; f02.m[a][a] = f02.m[a][a] + cd{0.0, e02};
      f03.m[a][a] = f03.m[a][a] + cd{0.0, e03}; f12.m[a][a] = f12.m[a][a] + cd{0.0, e12};
      f13.m[a][a] = f13.m[a][a] + cd{0.0, e13}; f23.m[a][a] = f23.m[a][a] + cd{0.0, e23};
    }
  }
  // Schroedinger-functional boundary improvement: + (c_F - 1) at x0 = 1, T-1
  if (g.bc_t == 0.f && (x[0] == 1 || x[0] == g.L[0] - 1)) c0 += cF - 1.0;
  const double h = 0.5;
  for (int b = 0; b < 2; ++b) {
    // X_k = (i c_sw/2) G_k, G_k = F_0k - Fd_k (b = 0) or -(F_0k + Fd_k) (b = 1)
    cd X[3][3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cd g1 = b == 0 ? f01.m[a][c] - f23.m[a][c] : -(f01.m[a][c] + f23.m[a][c]);
        cd g2 = b == 0 ? f02.m[a][c] + f13.m[a][c] : -(f02.m[a][c] - f13.m[a][c]);
        cd g3 = b == 0 ? f03.m[a][c] - f12.m[a][c] : -(f03.m[a][c] + f12.m[a][c]);
        X[0][a][c] = h * times_i(g1);
        X[1][a][c] = h * times_i(g2);
        X[2][a][c] = h * times_i(g3);
      }
    cd m[6][6], mi[6][6], w[6][6];
    // [[c0 + X3, X1 - i X2], [X1 + i X2, c0 - X3]]
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        cd id = cd{a == c ? c0 : 0.0, 0.0};
        m[a][c] = id + X[2][a][c];
        m[a][c + 3] = X[0][a][c] - times_i(X[1][a][c]);
        m[a + 3][c] = X[0][a][c] + times_i(X[1][a][c]);
        m[a + 3][c + 3] = id - X[2][a][c];
      }
    store_block(g, p, i, b, m, a64, a32);
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int c = 0; c < 6; ++c) w[r][c] = m[r][c];
    if (!invert6(w, mi)) atomicExch(status, 1);
    store_block(g, p, i, b, mi, i64, i32);
  }
}

cudaError_t build_clover(const Geom& g, const double* links, const double* au1, double q, int qed_split,
                         double kappa, double csw, double csw_qed, double cF, double* a64, float* a32,
                         double* i64, float* i32, int* status_dev, cudaStream_t s) {
  const double c0 = 1.0 / (2.0 * kappa);
  const int qed = au1 ? (qed_split ? 2 : 1) : 0;
  dim3 block(128), grid((unsigned)((g.Vh + 127) / 128), 2);
  clover_kernel<<<grid, block, 0, s>>>(g, reinterpret_cast<const double2*>(links), au1, q, qed, c0, csw, csw_qed, cF,
                                       reinterpret_cast<double2*>(a64), reinterpret_cast<float4*>(a32),
                                       reinterpret_cast<double2*>(i64), reinterpret_cast<float4*>(i32), status_dev);
  return cudaGetLastError();
}

}  // namespace oq
