// Krylov solvers of libhb (Eqs. (Axb2), (Axb3); solver settings of Sec. 4)
// and the excitation / far-field kernels.
//
//  HB_C128:  GMRES(restart) on  L~^{-1} A U~^{-1} y = L~^{-1} b,  x = U~^{-1} y,
//            all FP64; the true residual ||b - A x|| is checked at every restart.
//  HB_C64:   FP64 iterative refinement; each refinement step is one cycle of
//            flexible GMRES right-preconditioned by U~^{-1} L~^{-1}, with the
//            preconditioner, the operator and the Arnoldi basis in complex FP32
//            (Hessenberg, Givens and the iterate in FP64).  The residual
//            b - A x between steps is computed with FP64-accurate arithmetic
//            on the stored factors (double-float pairs of FP32 for 32 or more
//            columns, FP64 below) while any column is above 1e-3; below that
//            the small correction dz is applied in FP32 and r -= A dz
//            accumulated in FP64.
// Right-hand sides are solved together in lockstep (one Krylov space per
// column); reductions run in a fixed order, so results are bitwise repeatable.
// With two or more columns every restart cycle runs as one CUDA graph launch
// (the Arnoldi steps, their CGS2, the Givens rotations and the convergence test
// on the device; see record_cycle in hb_gmres); one column runs the
// host-driven loop, which takes the same steps with a host round trip each.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <functional>
#include <vector>

#include "hb_api_internal.h"
#include "hb_sweep_launch.h"

namespace hb {

using zc = std::complex<double>;

// ---------------------------------------------------------------------------
// BLAS-1 style kernels on [row][R] blocks (double2)
// ---------------------------------------------------------------------------
static constexpr int kRedBlocks = 304;   // 2 x 152 SMs
static constexpr int kRedThreads = 256;

// partial[v][blk][r] = sum over this block's rows of conj(V_v[row][r]) * w[row][r]
// (VT = double2: FP64 arithmetic; VT = float2: FP32 products and per-thread
// sums, FP64 from the block reduction on)
template <class VT>
__global__ void k_dots_partial(const VT* __restrict__ V, int64_t vstride, int nvec,
                               const VT* __restrict__ w, int64_t n, int64_t R, double2* __restrict__ partial) {
  using S = decltype(VT::x);
  __shared__ double2 red[kRedThreads];
  const int v = blockIdx.y;
  const VT* Vv = V + (int64_t)v * vstride;
  const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t row0 = (int64_t)blockIdx.x * rows_per, row1 = min(n, row0 + rows_per);
  const int G = (R >= kRedThreads) ? 1 : kRedThreads / (int)R;   // row groups
  for (int64_t rbase = 0; rbase < R; rbase += kRedThreads) {
    const int t = threadIdx.x;
    int64_t r = (R >= kRedThreads) ? rbase + t : t % R;
    int g = (R >= kRedThreads) ? 0 : t / (int)R;
    S ax = 0, ay = 0;
    if (g < G && r < R) {
      for (int64_t row = row0 + g; row < row1; row += G) {
        VT a = Vv[row * R + r], b = w[row * R + r];
        ax = fma(a.x, b.x, fma(a.y, b.y, ax));
        ay = fma(a.x, b.y, fma(-a.y, b.x, ay));
      }
    }
    red[t] = double2{(double)ax, (double)ay};
    __syncthreads();
    if (R >= kRedThreads) {
      if (r < R) partial[((int64_t)v * gridDim.x + blockIdx.x) * R + r] = red[t];
    } else if (t < R) {
      double2 s = {0.0, 0.0};
      for (int gg = 0; gg < G; ++gg) { s.x += red[gg * R + t].x; s.y += red[gg * R + t].y; }
      partial[((int64_t)v * gridDim.x + blockIdx.x) * R + t] = s;
    }
    __syncthreads();
    if (R < kRedThreads) break;
  }
}

// out[v][r] = sum_blk partial[v][blk][r] (fixed order)
__global__ void k_dots_final(const double2* __restrict__ partial, int nblk, int nvec, int64_t R, double2* out) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nvec * R) return;
  int v = (int)(e / R);
  int64_t r = e % R;
  double2 s = {0.0, 0.0};
  for (int b = 0; b < nblk; ++b) {
    double2 p = partial[((int64_t)v * nblk + b) * R + r];
    s.x += p.x;
    s.y += p.y;
  }
  out[e] = s;
}

// w[row][r] -= sum_v V_v[row][r] h[v][r]   (h and the arithmetic in the precision of VT)
template <class VT>
__global__ void k_sub_combo(const VT* __restrict__ V, int64_t vstride, int nvec, const VT* __restrict__ h,
                            VT* __restrict__ w, int64_t n, int64_t R) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < n * R; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e % R;
    VT acc = w[e];
    for (int v = 0; v < nvec; ++v) {
      const VT a = V[(int64_t)v * vstride + e], c = h[(int64_t)v * R + r];
      acc.x -= a.x * c.x - a.y * c.y;
      acc.y -= a.x * c.y + a.y * c.x;
    }
    w[e] = acc;
  }
}

// The first CGS2 pass's update fused with the second pass's dot products, for
// R >= kRedThreads (one thread per column): w[row][r] -= sum_v V_v[row][r] h[v][r],
// then partial[v][blk][r] = sum over the block's rows of conj(V_v[row][r]) w[row][r]
// with the updated w.  V is read once for both, instead of once by k_sub_combo and
// once by k_dots_partial; the arithmetic and the partial sums' row order are those
// two kernels'.  NV >= nvec (the vectors' values stay in registers).
template <class VT, int NV>
__global__ void __launch_bounds__(kRedThreads) k_sub_dots(const VT* __restrict__ V, int64_t vstride, int nvec,
                                                          const VT* __restrict__ h, VT* __restrict__ w, int64_t n,
                                                          int64_t R, double2* __restrict__ partial) {
  using S = decltype(VT::x);
  const int64_t r = (int64_t)blockIdx.y * blockDim.x + threadIdx.x;
  if (r >= R) return;
  const int64_t rows_per = (n + gridDim.x - 1) / gridDim.x;
  const int64_t row0 = (int64_t)blockIdx.x * rows_per, row1 = min(n, row0 + rows_per);
  VT hv[NV];
  S ax[NV], ay[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    hv[v] = v < nvec ? h[(int64_t)v * R + r] : VT{0, 0};
    ax[v] = 0;
    ay[v] = 0;
  }
  for (int64_t row = row0; row < row1; ++row) {
    const int64_t e = row * R + r;
    VT vv[NV];
#pragma unroll
    for (int v = 0; v < NV; ++v) vv[v] = v < nvec ? V[(int64_t)v * vstride + e] : VT{0, 0};
    VT acc = w[e];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if (v < nvec) {
        acc.x -= vv[v].x * hv[v].x - vv[v].y * hv[v].y;
        acc.y -= vv[v].x * hv[v].y + vv[v].y * hv[v].x;
      }
    }
    w[e] = acc;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      ax[v] = fma(vv[v].x, acc.x, fma(vv[v].y, acc.y, ax[v]));
      ay[v] = fma(vv[v].x, acc.y, fma(-vv[v].y, acc.x, ay[v]));
    }
  }
#pragma unroll
  for (int v = 0; v < NV; ++v)
    if (v < nvec) partial[((int64_t)v * gridDim.x + blockIdx.x) * R + r] = double2{(double)ax[v], (double)ay[v]};
}

// whether k_sub_dots serves nvec vectors of R columns (complex-FP32 bases: an FP64
// basis's values would not fit the registers), and its launch
template <class VT>
static inline bool sub_dots_ok(int nvec, int64_t R) { return sizeof(VT) == 8 && R >= kRedThreads && nvec <= 32; }
template <class VT>
static void launch_sub_dots(const VT* V, int64_t vstride, int nvec, const VT* h, VT* w, int64_t n, int64_t R,
                            double2* partial, cudaStream_t s) {
  if constexpr (sizeof(VT) == 8) {
    const dim3 grid(kRedBlocks, (unsigned)((R + kRedThreads - 1) / kRedThreads));
    if (nvec <= 8) k_sub_dots<VT, 8><<<grid, kRedThreads, 0, s>>>(V, vstride, nvec, h, w, n, R, partial);
    else if (nvec <= 16) k_sub_dots<VT, 16><<<grid, kRedThreads, 0, s>>>(V, vstride, nvec, h, w, n, R, partial);
    else k_sub_dots<VT, 32><<<grid, kRedThreads, 0, s>>>(V, vstride, nvec, h, w, n, R, partial);
  }
}

// dst[row][r] = src[row][r] * s[r]  (s real; src / dst double2 or float2)
template <class SRC, class DST>
__global__ void k_scale_cols(const SRC* __restrict__ src, const double* __restrict__ s, DST* dst, int64_t n,
                             int64_t R) {
  using S = decltype(DST::x);
  using SS = decltype(SRC::x);
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < n * R; e += (int64_t)gridDim.x * blockDim.x) {
    // in the narrower of the two precisions (FP32 vectors stay off the FP64 pipe)
    if (sizeof(S) < sizeof(SS)) {
      const S f = (S)s[e % R];
      dst[e] = {(S)src[e].x * f, (S)src[e].y * f};
    } else {
      const SS f = (SS)s[e % R];
      dst[e] = {(S)(src[e].x * f), (S)(src[e].y * f)};
    }
  }
}

// y[e] += x[e] (optionally x converted from float2)
template <class S>
__global__ void k_axpy1(const S* __restrict__ x, double2* __restrict__ y, int64_t total) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    y[e].x += (double)x[e].x;
    y[e].y += (double)x[e].y;
  }
}

// y[row][r] += sum_v Z_v[row][r] c[v][r]  (Z and c double2, or both float2: the
// combination is then formed in FP32 and added to the FP64 y once)
template <class S>
__global__ void k_add_combo(const S* __restrict__ Z, int64_t zstride, int nvec, const S* __restrict__ c,
                            double2* __restrict__ y, int64_t n, int64_t R) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < n * R; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e % R;
    S acc = {0, 0};
    for (int v = 0; v < nvec; ++v) {
      const S a = Z[(int64_t)v * zstride + e], cc = c[(int64_t)v * R + r];
      acc.x += a.x * cc.x - a.y * cc.y;
      acc.y += a.x * cc.y + a.y * cc.x;
    }
    y[e].x += (double)acc.x;
    y[e].y += (double)acc.y;
  }
}

// y[row][r] = x[row][r] + s[r] y[row][r]  (complex per-column s; TFQMR direction updates)
__global__ void k_xpay(const double2* __restrict__ x, const double2* __restrict__ s, double2* __restrict__ y,
                       int64_t n, int64_t R) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < n * R; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 c = s[e % R], yy = y[e], xx = x[e];
    y[e] = {xx.x + c.x * yy.x - c.y * yy.y, xx.y + c.x * yy.y + c.y * yy.x};
  }
}

// r[e] -= a[e]  (a complex FP32, r FP64)
__global__ void k_sub_f32(const float2* __restrict__ a, double2* __restrict__ r, int64_t total) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    r[e].x -= (double)a[e].x;
    r[e].y -= (double)a[e].y;
  }
}

__global__ void k_sub_into(const double2* __restrict__ a, const double2* __restrict__ b, double2* out, int64_t total) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < total; e += (int64_t)gridDim.x * blockDim.x) out[e] = {a[e].x - b[e].x, a[e].y - b[e].y};
}

__global__ void k_to_f32(const double2* __restrict__ a, float2* __restrict__ b, int64_t total) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < total; e += (int64_t)gridDim.x * blockDim.x) b[e] = {(float)a[e].x, (float)a[e].y};
}

__global__ void k_nonfinite(const double2* __restrict__ a, int64_t ld, int64_t n, int64_t R, int* flag) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < n * R; e += (int64_t)gridDim.x * blockDim.x) {
    double2 v = a[(e / n) * ld + e % n];
    if (!isfinite(v.x) || !isfinite(v.y)) atomicExch(flag, 1);
  }
}

// r(col-major) = b(col-major) - y([row][R])
__global__ void k_residual_cols(const double2* __restrict__ b, int64_t ld, const double2* __restrict__ y, int64_t n,
                                int64_t R, double2* __restrict__ r) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < n * R; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t row = e / R, c = e % R;
    double2 bb = b[c * ld + row], yy = y[e];
    r[c * ld + row] = {bb.x - yy.x, bb.y - yy.y};
  }
}

// max that keeps a NaN once seen (reports of diverged columns)
static inline double nan_max(double a, double b) { return (std::isnan(a) || std::isnan(b)) ? NAN : std::max(a, b); }

static inline int gsz(int64_t total) {
  int64_t g = (total + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, 152 * 16));
}

int launch_residual_cols(const void* b, int64_t ld, const void* y, int64_t n, int64_t R, void* r, cudaStream_t st) {
  k_residual_cols<<<gsz(n * R), 256, 0, st>>>((const double2*)b, ld, (const double2*)y, n, R, (double2*)r);
  return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ECUDA;
}

// ---------------------------------------------------------------------------
// Excitation and far field
// ---------------------------------------------------------------------------
__global__ void k_plane_wave(const double* __restrict__ cx, const double* __restrict__ cy, int64_t n,
                             const double* __restrict__ cphi, const double* __restrict__ sphi, int64_t R,
                             double kappa, double2* __restrict__ b, int64_t ld) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < n * R; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e / n, i = e % n;
    double ph = -kappa * (cx[i] * cphi[r] + cy[i] * sphi[r]);
    double s, c;
    sincos(ph, &s, &c);
    b[r * ld + i] = {c, s};
  }
}

// out[r][q] = C * sum_n w_n x_n exp(+i k (x_n cos phi_q + y_n sin phi_q)); one block per (q, r),
// fixed-order block reduction.
__global__ void k_far_field(const double* __restrict__ cx, const double* __restrict__ cy,
                            const double* __restrict__ w, int64_t n, const double2* __restrict__ x, int64_t ld,
                            const double* __restrict__ cphi, const double* __restrict__ sphi, int64_t nobs,
                            double kappa, double2 C, double2* __restrict__ out, int mono_sign) {
  __shared__ double2 red[256];
  const int64_t q = blockIdx.x, r = blockIdx.y;
  const double2* xr = x + r * ld;
  const int64_t qq = mono_sign ? r : q;
  double2 acc = {0.0, 0.0};
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double ph = kappa * (cx[i] * cphi[qq] + cy[i] * sphi[qq]);
    if (mono_sign) ph = -ph;   // backscatter: steering vector equals b_n
    double s, c;
    sincos(ph, &s, &c);
    double2 v = xr[i];
    acc.x += w[i] * (v.x * c - v.y * s);
    acc.y += w[i] * (v.x * s + v.y * c);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      red[threadIdx.x].x += red[threadIdx.x + off].x;
      red[threadIdx.x].y += red[threadIdx.x + off].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double2 s = red[0];
    out[r * (mono_sign ? 1 : nobs) + (mono_sign ? 0 : q)] = {C.x * s.x - C.y * s.y, C.x * s.y + C.y * s.x};
  }
}

// out[r][n] (col-major, ld) = conj(C) w_n sum_q exp(-i k (x_n cos phi_q + y_n sin phi_q)) g[r][q]
// (the conjugate transpose of the far-field map), one thread per (n, r), fixed-order sum over q.
__global__ void k_far_field_adj(const double* __restrict__ cx, const double* __restrict__ cy,
                                const double* __restrict__ w, int64_t n, const double2* __restrict__ g, int64_t nobs,
                                const double* __restrict__ cphi, const double* __restrict__ sphi, int64_t R,
                                double kappa, double2 Cc, double2* __restrict__ out, int64_t ld) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; e < n * R; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, r = e / n;
    double2 acc = {0.0, 0.0};
    for (int64_t q = 0; q < nobs; ++q) {
      double ph = -kappa * (cx[i] * cphi[q] + cy[i] * sphi[q]);
      double s, c;
      sincos(ph, &s, &c);
      double2 gv = g[r * nobs + q];
      acc.x += gv.x * c - gv.y * s;
      acc.y += gv.x * s + gv.y * c;
    }
    acc = {w[i] * acc.x, w[i] * acc.y};
    out[r * ld + i] = {Cc.x * acc.x - Cc.y * acc.y, Cc.x * acc.y + Cc.y * acc.x};
  }
}

// ---------------------------------------------------------------------------
// GMRES machinery
// ---------------------------------------------------------------------------
struct Dev {
  hb_factor_t f;
  cudaStream_t st;
  int64_t n, R;
  double2* red_partial;
  double2* red_out;
  double* scal;
};

// the partial dot products in d.red_partial reduced to hh[v*R + r] (host copy)
static int dots_finish(Dev& d, int nvec, std::vector<zc>& hh) {
  int64_t tot = (int64_t)nvec * d.R;
  k_dots_final<<<(unsigned)((tot + 255) / 256), 256, 0, d.st>>>(d.red_partial, kRedBlocks, nvec, d.R, d.red_out); count_launch(d.f, 1);
  hh.resize(tot);
  if (cudaMemcpyAsync(hh.data(), d.red_out, tot * sizeof(double2), cudaMemcpyDeviceToHost, d.st) != cudaSuccess)
    return HB_ECUDA;
  // the sweep kernels' bounded-wait flag travels with every reduction, so a
  // timed-out preconditioner stops the solver at its next synchronisation
  int herr = 0;
  GridBar* gb = (GridBar*)d.f->df.bar;
  if (cudaMemcpyAsync(&herr, &gb->err, sizeof(int), cudaMemcpyDeviceToHost, d.st) != cudaSuccess) return HB_ECUDA;
  if (cudaStreamSynchronize(d.st) != cudaSuccess) return HB_ECUDA;
  if (herr) {
    cudaMemsetAsync(&gb->err, 0, sizeof(int), d.st);   // reported here: later calls start clean
    set_error("a bounded device-side wait expired in a sweep kernel during the solve");
    return HB_ETIMEOUT;
  }
  return HB_OK;
}

// h[v][r] = <V_v, w>_r for v < nvec (host copy returned in hh[v*R + r])
template <class VT>
static int dots(Dev& d, const VT* V, int64_t vstride, int nvec, const VT* w, std::vector<zc>& hh) {
  dim3 grid(kRedBlocks, nvec);
  k_dots_partial<VT><<<grid, kRedThreads, 0, d.st>>>(V, vstride, nvec, w, d.n, d.R, d.red_partial); count_launch(d.f, 1);
  return dots_finish(d, nvec, hh);
}

// CGS2: orthogonalise w against V_0..V_{nvec-1}; returns h (nvec x R) and ||w|| (R).
template <class VT>
static int cgs2(Dev& d, const VT* V, int64_t vstride, int nvec, VT* w, std::vector<zc>& h,
                std::vector<double>& nrm) {
  std::vector<zc> h1, h2;
  int rc;
  h.assign((size_t)nvec * d.R, zc(0.0));
  // with k_sub_dots the first pass's update also forms the second pass's dot products
  const bool fused = sub_dots_ok<VT>(nvec, d.R);
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 0 || !fused) {
      if ((rc = dots(d, V, vstride, nvec, w, pass ? h2 : h1))) return rc;
    } else if ((rc = dots_finish(d, nvec, h2))) {
      return rc;
    }
    std::vector<zc>& hp = pass ? h2 : h1;
    for (size_t i = 0; i < h.size(); ++i) h[i] += hp[i];
    // the coefficients in the vectors' precision (converted once, on the host)
    std::vector<VT> hv(hp.size());
    for (size_t i = 0; i < hp.size(); ++i) hv[i] = VT{(decltype(VT::x))hp[i].real(), (decltype(VT::x))hp[i].imag()};
    if (cudaMemcpyAsync(d.red_out, hv.data(), hv.size() * sizeof(VT), cudaMemcpyHostToDevice, d.st) != cudaSuccess)
      return HB_ECUDA;
    if (pass == 0 && fused) {
      launch_sub_dots<VT>(V, vstride, nvec, (const VT*)d.red_out, w, d.n, d.R, d.red_partial, d.st);
    } else {
      k_sub_combo<VT><<<gsz(d.n * d.R), 256, 0, d.st>>>(V, vstride, nvec, (const VT*)d.red_out, w, d.n, d.R);
    }
    count_launch(d.f, 1);
  }
  std::vector<zc> nn;
  if ((rc = dots(d, w, 0, 1, w, nn))) return rc;
  nrm.resize(d.R);
  for (int64_t r = 0; r < d.R; ++r) nrm[r] = std::sqrt(std::max(nn[r].real(), 0.0));
  return HB_OK;
}

template <class VT>
static int norms(Dev& d, const VT* w, std::vector<double>& nrm) {
  std::vector<zc> nn;
  int rc = dots(d, w, 0, 1, w, nn);
  if (rc) return rc;
  nrm.resize(d.R);
  for (int64_t r = 0; r < d.R; ++r) nrm[r] = std::sqrt(std::max(nn[r].real(), 0.0));
  return HB_OK;
}

// dst = src / nrm (per column; zero-norm columns copied unchanged)
template <class SRC, class DST>
static void normalise(Dev& d, const SRC* src, const std::vector<double>& nrm, DST* dst) {
  std::vector<double> inv(d.R);
  for (int64_t r = 0; r < d.R; ++r) inv[r] = nrm[r] > 0 ? 1.0 / nrm[r] : 1.0;
  cudaMemcpyAsync(d.scal, inv.data(), d.R * sizeof(double), cudaMemcpyHostToDevice, d.st);
  k_scale_cols<SRC, DST><<<gsz(d.n * d.R), 256, 0, d.st>>>(src, d.scal, dst, d.n, d.R); count_launch(d.f, 1);
}

// Per-RHS Givens state of one restart cycle.
struct Givens {
  int m;
  std::vector<zc> H, cs, sn, g;    // H column-major (m+1) x m
  void reset(int mm, double beta) {
    m = mm;
    H.assign((size_t)(m + 1) * m, zc(0.0));
    cs.assign(m, zc(0.0));
    sn.assign(m, zc(0.0));
    g.assign(m + 1, zc(0.0));
    g[0] = beta;
  }
  // insert column j (entries h[0..j], hnext) and return |g_{j+1}|
  double push(int j, const zc* h, double hnext) {
    for (int i = 0; i <= j; ++i) H[(size_t)j * (m + 1) + i] = h[i];
    H[(size_t)j * (m + 1) + j + 1] = hnext;
    zc* col = &H[(size_t)j * (m + 1)];
    for (int i = 0; i < j; ++i) {   // G_i = [[c*, s*], [-s, c]]
      zc t = std::conj(cs[i]) * col[i] + std::conj(sn[i]) * col[i + 1];
      col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
      col[i] = t;
    }
    zc a = col[j], b = col[j + 1];
    double den = std::sqrt(std::norm(a) + std::norm(b));
    cs[j] = den > 0 ? a / den : zc(1.0);
    sn[j] = den > 0 ? b / den : zc(0.0);
    col[j] = std::conj(cs[j]) * a + std::conj(sn[j]) * b;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = std::conj(cs[j]) * g[j];
    return std::abs(g[j + 1]);
  }
  void solve(int k, zc* coef) const {
    for (int i = k - 1; i >= 0; --i) {
      zc acc = g[i];
      for (int l = i + 1; l < k; ++l) acc -= H[(size_t)l * (m + 1) + i] * coef[l];
      coef[i] = acc / H[(size_t)i * (m + 1) + i];
    }
  }
};

// ---------------------------------------------------------------------------
// Restart cycle on the device (graph mode of hb_gmres).  The Arnoldi steps,
// their CGS2 coefficients, the Givens rotations of every column's Hessenberg
// matrix, the convergence test and the least-squares solve all stay on the
// device, so that a whole cycle is one CUDA graph launch.  Every step is a
// chain of conditional (IF) nodes; step j's convergence test sets step j+1's
// conditions, so the steps after the last one needed do not run at all.  The
// arithmetic is the host loop's (FP64 Givens, CGS2 in the basis precision
// with FP64 reductions in the same fixed order).
// ---------------------------------------------------------------------------
struct Cyc {
  int64_t R;
  int m;
  double2* H;       // [R][m][m+1]: column j of column c's Hessenberg matrix at H + (c m + j)(m + 1)
  double2* cs;      // [R][m] rotations
  double2* sn;      // [R][m]
  double2* g;       // [R][m+1] rotated right-hand side beta e_1
  double2* hacc;    // [m+1][R] CGS2 coefficients of the current step (sum of both passes)
  void* cvec;       // [m+1][R] one pass's coefficients in the basis precision
  double* hn;       // [R] ||w|| after CGS2
  double* inv;      // [R] 1 / ||w|| (1 for a zero column)
  const double* prm;   // [4][R] host-written per cycle: target = max(t_abs, t_rel beta); bnorm; skip
  double* pres;     // [R] preconditioned estimate / ||b||
  double* target;   // [R]
  int* kuse;        // [R] 0 active, 1 not in this cycle, -(j+1) converged after step j+1
  int* ctl;         // [0] step limit (host-written), [1] steps run
};

// the conditions of the next step's IF nodes (n = 0 after the last step)
constexpr int kMaxSeg = 6;
struct CondNext {
  cudaGraphConditionalHandle h[kMaxSeg];
  int n;
};

__device__ __forceinline__ double2 z_mul(double2 a, double2 b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ double2 z_cmul(double2 a, double2 b) {   // conj(a) b
  return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}

// beta = ||r|| per column (the fixed-order sum of the partial dot products),
// 1 / beta for the start vector, g = beta e_1, the column's target and state
__global__ void k_cyc_start(const double2* __restrict__ partial, int nblk, Cyc c) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= c.R) return;
  double2 sum = {0.0, 0.0};
  for (int b = 0; b < nblk; ++b) {
    const double2 p = partial[(int64_t)b * c.R + col];
    sum.x += p.x;
    sum.y += p.y;
  }
  const double beta = sqrt(fmax(sum.x, 0.0));
  c.inv[col] = beta > 0 ? 1.0 / beta : 1.0;
  c.g[col * (c.m + 1)] = {beta, 0.0};
  c.target[col] = fmax(c.prm[col], c.prm[c.R + col] * beta);
  c.kuse[col] = c.prm[3 * c.R + col] != 0.0 ? 1 : 0;
}

// one CGS2 pass's coefficients: hacc (+)= <V_v, w>, cvec = the same in the basis precision
template <class VT>
__global__ void k_cgs_final(const double2* __restrict__ partial, int nblk, int nvec, Cyc c, int pass) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nvec * c.R) return;
  const int v = (int)(e / c.R);
  const int64_t r = e % c.R;
  double2 sum = {0.0, 0.0};
  for (int b = 0; b < nblk; ++b) {
    const double2 p = partial[((int64_t)v * nblk + b) * c.R + r];
    sum.x += p.x;
    sum.y += p.y;
  }
  double2 h = sum;
  if (pass) h = {c.hacc[e].x + sum.x, c.hacc[e].y + sum.y};
  c.hacc[e] = h;
  ((VT*)c.cvec)[e] = VT{(decltype(VT::x))sum.x, (decltype(VT::x))sum.y};
}

// ||w|| and 1 / ||w|| per column
__global__ void k_norm_final(const double2* __restrict__ partial, int nblk, Cyc c) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= c.R) return;
  double2 sum = {0.0, 0.0};
  for (int b = 0; b < nblk; ++b) {
    const double2 p = partial[(int64_t)b * c.R + col];
    sum.x += p.x;
    sum.y += p.y;
  }
  const double nrm = sqrt(fmax(sum.x, 0.0));
  c.hn[col] = nrm;
  c.inv[col] = nrm > 0 ? 1.0 / nrm : 1.0;
}

// Step j of every active column: insert the new Hessenberg column, apply the
// earlier rotations, form and apply rotation j (G = [[c*, s*], [-s, c]]), and
// test |g_{j+1}| against the column's target; one CTA, columns strided over its
// threads.  Thread 0 records the step count and sets the next step's
// conditions: 1 while some column is active and the step limit allows.
__global__ void k_givens(Cyc c, int j, CondNext nx) {
  const int m = c.m;
  int active = 0;
  for (int64_t col = threadIdx.x; col < c.R; col += blockDim.x) {
    if (c.kuse[col] != 0) continue;
    double2* h = c.H + ((size_t)col * m + j) * (m + 1);
    for (int i = 0; i <= j; ++i) h[i] = c.hacc[(size_t)i * c.R + col];
    h[j + 1] = {c.hn[col], 0.0};
    double2* cs = c.cs + (size_t)col * m;
    double2* sn = c.sn + (size_t)col * m;
    for (int i = 0; i < j; ++i) {
      const double2 a = h[i], b = h[i + 1];
      const double2 t0 = z_cmul(cs[i], a), t1 = z_cmul(sn[i], b);
      const double2 u0 = z_mul(sn[i], a), u1 = z_mul(cs[i], b);
      h[i] = {t0.x + t1.x, t0.y + t1.y};
      h[i + 1] = {u1.x - u0.x, u1.y - u0.y};
    }
    const double2 a = h[j], b = h[j + 1];
    const double den = sqrt((a.x * a.x + a.y * a.y) + (b.x * b.x + b.y * b.y));
    const double2 cj = den > 0 ? double2{a.x / den, a.y / den} : double2{1.0, 0.0};
    const double2 sj = den > 0 ? double2{b.x / den, b.y / den} : double2{0.0, 0.0};
    cs[j] = cj;
    sn[j] = sj;
    const double2 t0 = z_cmul(cj, a), t1 = z_cmul(sj, b);
    h[j] = {t0.x + t1.x, t0.y + t1.y};
    h[j + 1] = {0.0, 0.0};
    double2* g = c.g + (size_t)col * (m + 1);
    const double2 gj = g[j], sg = z_mul(sj, gj);
    g[j + 1] = {-sg.x, -sg.y};
    g[j] = z_cmul(cj, gj);
    const double est = hypot(g[j + 1].x, g[j + 1].y);
    const double bn = c.prm[2 * c.R + col];
    c.pres[col] = bn > 0 ? est / bn : 0.0;
    if (est <= c.target[col]) c.kuse[col] = -(j + 1);
    else active = 1;
  }
  active = __syncthreads_or(active);
  if (threadIdx.x == 0) {
    c.ctl[1] = j + 1;
    const unsigned go = (active && j + 1 < c.ctl[0]) ? 1u : 0u;
    for (int k = 0; k < nx.n; ++k) cudaGraphSetConditional(nx.h[k], go);
  }
}

// After the cycle: each column's least-squares solution by back substitution
// over its own step count, written as the combination coefficients coef[i][c]
// (basis precision) of the steps that ran; columns outside the cycle get
// zeros.  y: [m][R] FP64 scratch.
template <class VT>
__global__ void k_cyc_solve(Cyc c, double2* __restrict__ y, VT* __restrict__ coef) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= c.R) return;
  const int m = c.m, kc = c.ctl[1];
  const int ku = c.kuse[col];
  const int k = ku == 1 ? 0 : (ku < 0 ? -ku : kc);
  const double2* H = c.H + (size_t)col * m * (m + 1);
  const double2* g = c.g + (size_t)col * (m + 1);
  for (int i = k - 1; i >= 0; --i) {
    double2 acc = g[i];
    for (int l = i + 1; l < k; ++l) {
      const double2 p = z_mul(H[(size_t)l * (m + 1) + i], y[(size_t)l * c.R + col]);
      acc = {acc.x - p.x, acc.y - p.y};
    }
    const double2 d = H[(size_t)i * (m + 1) + i];
    const double dd = d.x * d.x + d.y * d.y;
    y[(size_t)i * c.R + col] = {(acc.x * d.x + acc.y * d.y) / dd, (acc.y * d.x - acc.x * d.y) / dd};
  }
  using S = decltype(VT::x);
  for (int i = 0; i < kc; ++i) {
    const double2 v = i < k ? y[(size_t)i * c.R + col] : double2{0.0, 0.0};
    coef[(size_t)i * c.R + col] = VT{(S)v.x, (S)v.y};
  }
}

// CGS2 of step nvec-1 of a captured cycle: two passes (coefficients reduced on
// the device in fixed order, accumulated in FP64), then ||w|| and w / ||w||.
template <class VT>
static void cgs2_graph(hb_factor_t f, const Dev& d, const Cyc& cyc, const VT* V, int nvec, VT* w, cudaStream_t s) {
  const int64_t nR = d.n * d.R;
  const bool fused = sub_dots_ok<VT>(nvec, d.R);   // the first update forms the second pass's dot products
  const unsigned gfin = (unsigned)(((int64_t)nvec * d.R + 255) / 256);
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 0 || !fused)
      k_dots_partial<VT><<<dim3(kRedBlocks, nvec), kRedThreads, 0, s>>>(V, nR, nvec, w, d.n, d.R, d.red_partial);
    k_cgs_final<VT><<<gfin, 256, 0, s>>>(d.red_partial, kRedBlocks, nvec, cyc, pass);
    if (pass == 0 && fused)
      launch_sub_dots<VT>(V, nR, nvec, (const VT*)cyc.cvec, w, d.n, d.R, d.red_partial, s);
    else
      k_sub_combo<VT><<<gsz(nR), 256, 0, s>>>(V, nR, nvec, (const VT*)cyc.cvec, w, d.n, d.R);
  }
  k_dots_partial<VT><<<dim3(kRedBlocks, 1), kRedThreads, 0, s>>>(w, 0, 1, w, d.n, d.R, d.red_partial);
  k_norm_final<<<(unsigned)((d.R + 255) / 256), 256, 0, s>>>(d.red_partial, kRedBlocks, cyc);
  k_scale_cols<VT, VT><<<gsz(nR), 256, 0, s>>>(w, cyc.inv, w, d.n, d.R);
  count_launch(f, fused ? 8 : 9);
}

}  // namespace hb

using namespace hb;

extern "C" int hb_gmres(hb_factor_t f, int op, const void* b_phys, void* x, int64_t nrhs, int64_t ld, int restart,
                        double rtol, int maxit, hb_gmres_info* info, void* stream) {
  int rc = check_vec_args(f, b_phys, x, nrhs, ld, "hb_gmres");
  if (rc) return rc;
  if (op != HB_OP_N && op != HB_OP_H) { set_error("hb_gmres: bad op"); return HB_EINVAL; }
  if (restart < 1 || restart > 512 || !(rtol > 0) || maxit < 1) { set_error("hb_gmres: bad restart/rtol/maxit"); return HB_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  auto t0 = std::chrono::steady_clock::now();
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("hb_gmres: stream error"); return HB_ECUDA; }
  const DevFactor& df = f->df;
  const int64_t n = df.n, R = nrhs;
  const bool adj = op == HB_OP_H;
  const bool mixed = df.form != HB_C128;
  const int m = restart;
  const size_t vbytes = (size_t)n * R * sizeof(double2);
  Workspace& ws = f->ws;
  double2* bh = (double2*)ws.get(WS_VEC2, vbytes);            // scaled b (internal layout)
  double2* xv = (double2*)ws.get(WS_VEC3, vbytes);            // x (split form: y) iterate
  // Krylov basis: FP64 for HB_C128; complex FP32 for the FP32 forms (the inner
  // FGMRES of the refinement loop; the residual between steps stays FP64)
  const size_t vbytes_basis = mixed ? (size_t)n * R * sizeof(float2) : vbytes;
  void* Vb = ws.get(WS_BASIS, vbytes_basis * (m + 1));
  double2* V = (double2*)Vb;
  float2* V32 = (float2*)Vb;
  double2* red = (double2*)ws.get(WS_RED, (size_t)kRedBlocks * (m + 2) * R * sizeof(double2) + (size_t)(m + 2) * R * sizeof(double2) + R * sizeof(double));
  void* zb = mixed ? ws.get(WS_ZBASIS, (size_t)n * R * sizeof(float2) * (m + 1)) : nullptr;   // FGMRES Z (float2) + f32 scratch
  int* flag = (int*)ws.get(WS_SMALL, 256);
  if (!bh || !xv || !Vb || !red || !flag || (mixed && !zb)) { set_error("hb_gmres: workspace allocation failed"); return HB_ENOMEM; }
  double2* tmp = (double2*)ws.get(WS_VEC0, vbytes);
  double2* tmp2 = (double2*)ws.get(WS_VEC1, vbytes);
  if (!tmp || !tmp2) { set_error("hb_gmres: workspace allocation failed"); return HB_ENOMEM; }
  Dev d{f, st, n, R, red, red + (size_t)kRedBlocks * (m + 2) * R, (double*)(red + (size_t)kRedBlocks * (m + 2) * R + (size_t)(m + 2) * R)};

  // graph mode: the device-side cycle state, and every workspace that the
  // captured kernels or the steps between cycles use reserved at its largest
  // size first, so that no allocation moves a buffer the graph holds
  bool use_graph = f->gmres_graph != 0 && R >= 2;
  Cyc cyc{};
  double2* ysolve = nullptr;
  void* coefd = nullptr;
  if (use_graph) {
    const size_t R_ = (size_t)R, m_ = (size_t)m;
    const size_t parts[] = {R_ * m_ * (m_ + 1) * 16, R_ * m_ * 16, R_ * m_ * 16, R_ * (m_ + 1) * 16, (m_ + 1) * R_ * 16,
                            (m_ + 1) * R_ * 16, R_ * 8, R_ * 8, 4 * R_ * 8, R_ * 8, R_ * 8, R_ * 4, 16, m_ * R_ * 16,
                            m_ * R_ * 16};
    size_t off[15], tot = 0;
    for (int i = 0; i < 15; ++i) { off[i] = tot; tot += (parts[i] + 255) / 256 * 256; }
    char* cb = (char*)ws.get(WS_CYC, tot);
    const int es_sweep = mixed ? 8 : 16;
    size_t sweep_need = (size_t)df.state_len * R * es_sweep;
    if (df.sw[0].ok) sweep_need = std::max(sweep_need, (size_t)sweep_cols_state_entries(df, R) * 8);
    const bool dd = mixed && apply_dd_ready(R);
    if (!cb || !ws.get(WS_STATE, (size_t)df.state_len * R * 16) || !ws.get(WS_STATE_SWEEP, sweep_need) ||
        (dd && (!ws.get(WS_DD0, (size_t)n * R * 16) || !ws.get(WS_DD1, (size_t)n * R * 16)))) {
      set_error("hb_gmres: workspace allocation failed");
      return HB_ENOMEM;
    }
    cyc.R = R;
    cyc.m = m;
    cyc.H = (double2*)(cb + off[0]);
    cyc.cs = (double2*)(cb + off[1]);
    cyc.sn = (double2*)(cb + off[2]);
    cyc.g = (double2*)(cb + off[3]);
    cyc.hacc = (double2*)(cb + off[4]);
    cyc.cvec = cb + off[5];
    cyc.hn = (double*)(cb + off[6]);
    cyc.inv = (double*)(cb + off[7]);
    cyc.prm = (const double*)(cb + off[8]);
    cyc.pres = (double*)(cb + off[9]);
    cyc.target = (double*)(cb + off[10]);
    cyc.kuse = (int*)(cb + off[11]);
    cyc.ctl = (int*)(cb + off[12]);
    ysolve = (double2*)(cb + off[13]);
    coefd = cb + off[14];
  }

  // non-finite input check
  cudaMemsetAsync(flag, 0, sizeof(int), st);
  k_nonfinite<<<gsz(n * R), 256, 0, st>>>((const double2*)b_phys, ld, n, R, flag); count_launch(f, 1);
  int hflag = 0;
  cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("hb_gmres: CUDA error"); return HB_ECUDA; }
  if (hflag) { set_error("hb_gmres: right-hand side contains NaN/Inf"); return HB_ENAN; }

  if ((rc = launch_gather_cols(b_phys, 0, ld, n, R, bh, 0, df.scale, st))) return rc;
  cudaMemsetAsync(xv, 0, vbytes, st);
  std::vector<double> bnorm;
  if ((rc = norms(d, bh, bnorm))) return rc;

  const Prec pres = mixed ? PREC_F32_ACC64 : PREC_F64;    // true residual precision
  const int lo = adj ? 3 : 0, up = adj ? 2 : 1;            // first / second sweep of M^{-1} (op N: L then U)
  // split form for op H solves A^H x = b: (U~^H)^{-1}... with A^H = U~^H... the split
  // system uses  L' = U~^H (lower) and U' = L~^H (upper):  U~^{-H} A^H L~^{-H}.
  int iters = 0, cycles = 0, nconv = 0;
  std::vector<int32_t> it_r(R, 0);
  std::vector<double> res_r(R, 1.0), pres_r(R, 0.0), tscale(R, 1.0);
  std::vector<char> done(R, 0);
  std::vector<Givens> gv(R);
  std::vector<zc> h;
  std::vector<double> hn;
  std::vector<int> kuse(R, 0);
  std::vector<zc> coef((size_t)m * R);
  float2* zf = (float2*)zb;                                     // Z_0..Z_{m-1} then a float2 scratch at Z_m
  float2* f32s = mixed ? zf + (size_t)m * n * R : nullptr;

  // r = b^ - A^ x  (FP64); returns per-column relative norms in res_r
  auto true_residual = [&](const double2* xx, double2* r) -> int {
    int e;
    if ((e = apply_internal(f, pres, adj, xx, tmp2, R, st))) return e;
    k_sub_into<<<gsz(n * R), 256, 0, st>>>(bh, tmp2, r, n * R); count_launch(f, 1);
    std::vector<double> rn;
    if ((e = norms(d, r, rn))) return e;
    for (int64_t c = 0; c < R; ++c) res_r[c] = bnorm[c] > 0 ? rn[c] / bnorm[c] : 0.0;
    return HB_OK;
  };

  // split form: x = U'^{-1} y ; preconditioned residual L'^{-1} r
  double2* r = tmp;   // residual / work vector
  // x = 0: r = b^ (no operator application needed)
  cudaMemcpyAsync(r, bh, vbytes, cudaMemcpyDeviceToDevice, st);
  for (int64_t c = 0; c < R; ++c) res_r[c] = bnorm[c] > 0 ? 1.0 : 0.0;

  // ---- graph mode: one restart cycle captured on stream s.  Each Arnoldi step
  // is a chain of IF nodes, one per segment (a copy, a sweep, the operator,
  // CGS2 + the Givens step), each body captured on stream sb.  Step 0's
  // conditions default to 1 at every launch, the others' to 0; step j's
  // Givens kernel sets step j+1's.  A conditional body holds no event nodes,
  // so the timing events (when profiling) sit between the IF nodes, tagged
  // with the step and read only for the steps that ran.
  const int64_t nR = n * R;
  const unsigned gcol = (unsigned)((R + 255) / 256);
  const int nseg = mixed ? 5 : 6;
  std::vector<cudaGraphConditionalHandle> hnd;
  auto record_cycle = [&](cudaStream_t s, cudaStream_t sb) -> int {
    cudaStreamCaptureStatus cst;
    cudaGraph_t g = nullptr;
    if (cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, nullptr, nullptr, nullptr) != cudaSuccess || !g) return HB_ECUDA;
    hnd.assign((size_t)m * nseg, cudaGraphConditionalHandle{});
    for (int j = 0; j < m; ++j)
      for (int k = 0; k < nseg; ++k)
        if (cudaGraphConditionalHandleCreate(&hnd[(size_t)j * nseg + k], g, j == 0 ? 1u : 0u,
                                             cudaGraphCondAssignDefault) != cudaSuccess)
          return HB_ECUDA;
    int e;
    f->prof.tag = -1;
    // start vector v_0 = r / ||r|| (split form: r <- L'^{-1} r first), g = beta e_1
    if (!mixed && (e = sweep_internal(f, PREC_F64, lo, r, R, s))) return e;
    k_dots_partial<double2><<<dim3(kRedBlocks, 1), kRedThreads, 0, s>>>(r, 0, 1, r, n, R, d.red_partial);
    k_cyc_start<<<gcol, 256, 0, s>>>(d.red_partial, kRedBlocks, cyc);
    if (mixed) k_scale_cols<double2, float2><<<gsz(nR), 256, 0, s>>>(r, cyc.inv, V32, n, R);
    else k_scale_cols<double2, double2><<<gsz(nR), 256, 0, s>>>(r, cyc.inv, V, n, R);
    count_launch(f, 3);
    // segment k of step j: an IF node on its condition; kind 0 / 1 (apply / sweep) gets timing events
    int seg_k = 0;
    auto segment = [&](int j, int kind, const std::function<int(cudaStream_t)>& body) -> int {
      const int k = seg_k++;
      cudaEvent_t ea = nullptr, eb = nullptr;
      if (f->prof.on && kind >= 0) {
        if (cudaEventCreate(&ea) != cudaSuccess) return HB_ECUDA;
        if (cudaEventCreate(&eb) != cudaSuccess) { cudaEventDestroy(ea); return HB_ECUDA; }
        f->prof.cap.push_back({kind, j, ea, eb});
        if (cudaEventRecordWithFlags(ea, s, cudaEventRecordExternal) != cudaSuccess) return HB_ECUDA;
      }
      const cudaGraphNode_t* deps = nullptr;
      size_t nd = 0;
      if (cudaStreamGetCaptureInfo(s, &cst, nullptr, &g, &deps, nullptr, &nd) != cudaSuccess) return HB_ECUDA;
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = hnd[(size_t)j * nseg + k];
      np.conditional.type = cudaGraphCondTypeIf;
      np.conditional.size = 1;
      cudaGraphNode_t node = nullptr;
      if (cudaGraphAddNode(&node, g, deps, nullptr, nd, &np) != cudaSuccess) return HB_ECUDA;
      if (cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
        return HB_ECUDA;
      if (cudaStreamBeginCaptureToGraph(sb, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                        cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return HB_ECUDA;
      f->prof.in_body = true;
      const int be = body(sb);
      f->prof.in_body = false;
      cudaGraph_t bg = nullptr;
      const cudaError_t ce = cudaStreamEndCapture(sb, &bg);
      if (be) return be;
      if (ce != cudaSuccess) return HB_ECUDA;
      if (eb && cudaEventRecordWithFlags(eb, s, cudaEventRecordExternal) != cudaSuccess) return HB_ECUDA;
      return HB_OK;
    };
    for (int j = 0; j < m; ++j) {
      f->prof.tag = j;
      seg_k = 0;
      CondNext nx{};
      nx.n = j + 1 < m ? nseg : 0;
      for (int k = 0; k < nx.n; ++k) nx.h[k] = hnd[(size_t)(j + 1) * nseg + k];
      if (mixed) {   // z_j = M^{-1} v_j, w = A z_j (complex FP32)
        float2* zj = zf + (size_t)j * nR;
        float2* w32 = V32 + (size_t)(j + 1) * nR;
        const float2* vj = V32 + (size_t)j * nR;
        if ((e = segment(j, -1, [&](cudaStream_t b) {
               return cudaMemcpyAsync(zj, vj, (size_t)nR * sizeof(float2), cudaMemcpyDeviceToDevice, b) == cudaSuccess
                          ? HB_OK : HB_ECUDA; })))
          return e;
        if ((e = segment(j, 1, [&](cudaStream_t b) { return sweep_internal(f, PREC_F32, lo, zj, R, b); }))) return e;
        if ((e = segment(j, 1, [&](cudaStream_t b) { return sweep_internal(f, PREC_F32, up, zj, R, b); }))) return e;
        if ((e = segment(j, 0, [&](cudaStream_t b) { return apply_internal(f, PREC_F32, adj, zj, w32, R, b); })))
          return e;
        if ((e = segment(j, -1, [&](cudaStream_t b) {
               cgs2_graph(f, d, cyc, (const float2*)V32, j + 1, w32, b);
               k_givens<<<1, 256, 0, b>>>(cyc, j, nx);
               count_launch(f, 1);
               return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ECUDA; })))
          return e;
      } else {       // w = L'^{-1} A U'^{-1} v_j
        double2* vj = V + (size_t)j * nR;
        double2* w = V + (size_t)(j + 1) * nR;
        if ((e = segment(j, -1, [&](cudaStream_t b) {
               return cudaMemcpyAsync(w, vj, vbytes, cudaMemcpyDeviceToDevice, b) == cudaSuccess ? HB_OK : HB_ECUDA; })))
          return e;
        if ((e = segment(j, 1, [&](cudaStream_t b) { return sweep_internal(f, PREC_F64, up, w, R, b); }))) return e;
        if ((e = segment(j, 0, [&](cudaStream_t b) { return apply_internal(f, PREC_F64, adj, w, tmp2, R, b); })))
          return e;
        if ((e = segment(j, -1, [&](cudaStream_t b) {
               return cudaMemcpyAsync(w, tmp2, vbytes, cudaMemcpyDeviceToDevice, b) == cudaSuccess ? HB_OK : HB_ECUDA; })))
          return e;
        if ((e = segment(j, 1, [&](cudaStream_t b) { return sweep_internal(f, PREC_F64, lo, w, R, b); }))) return e;
        if ((e = segment(j, -1, [&](cudaStream_t b) {
               cgs2_graph(f, d, cyc, (const double2*)V, j + 1, w, b);
               k_givens<<<1, 256, 0, b>>>(cyc, j, nx);
               count_launch(f, 1);
               return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ECUDA; })))
          return e;
      }
    }
    f->prof.tag = -1;
    if (mixed) k_cyc_solve<float2><<<gcol, 256, 0, s>>>(cyc, ysolve, (float2*)coefd);
    else k_cyc_solve<double2><<<gcol, 256, 0, s>>>(cyc, ysolve, (double2*)coefd);
    count_launch(f, 1);
    return cudaGetLastError() == cudaSuccess ? HB_OK : HB_ECUDA;
  };
  auto capture_cycle = [&]() -> int {
    f->cg.release(f->prof);
    cudaStream_t cs = nullptr, cb = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cb, cudaStreamNonBlocking) != cudaSuccess) {
      if (cs) cudaStreamDestroy(cs);
      set_error("hb_gmres: cannot create the capture streams");
      return HB_ECUDA;
    }
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
      cudaStreamDestroy(cs);
      cudaStreamDestroy(cb);
      set_error("hb_gmres: cannot begin the graph capture");
      return HB_ECUDA;
    }
    f->prof.capturing = true;
    f->prof.cap_launches.clear();
    int e = record_cycle(cs, cb);
    f->prof.capturing = false;
    f->prof.in_body = false;
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &g);
    cudaStreamDestroy(cs);
    cudaStreamDestroy(cb);
    cudaGraphExec_t ge = nullptr;
    cudaError_t ie = cudaSuccess;
    if (!e && (ce != cudaSuccess || !g || (ie = cudaGraphInstantiate(&ge, g, 0)) != cudaSuccess)) e = HB_ECUDA;
    if (e) {
      if (g) cudaGraphDestroy(g);
      f->prof.drop_capture();
      cudaGetLastError();
      set_error("hb_gmres: capturing the restart cycle as a CUDA graph failed (%s / %s)", cudaGetErrorString(ce),
                cudaGetErrorString(ie));
      return e;
    }
    CycleGraph& cg = f->cg;
    cg.graph = g;
    cg.exec = ge;
    cg.op = op;
    cg.R = R;
    cg.m = m;
    cg.mixed = mixed ? 1 : 0;
    cg.stamp = f->stamp;
    for (int i = 0; i < kSlots; ++i) cg.ws[i] = ws.ptr[i];
    return HB_OK;
  };
  std::vector<double> prm_h(4 * R), pres_h(R);
  std::vector<int> kuse_h(R);
  int graph_launches = 0;
  // one cycle: per-column targets in, graph launch, step count / states / estimates out
  auto graph_fresh = [&]() -> bool {
    const CycleGraph& cg = f->cg;
    bool fresh = cg.exec && cg.op == op && cg.R == R && cg.m == m && cg.mixed == (mixed ? 1 : 0) &&
                 cg.stamp == f->stamp;
    for (int i = 0; fresh && i < kSlots; ++i) fresh = cg.ws[i] == ws.ptr[i];
    return fresh;
  };
  auto graph_cycle = [&](int& kcyc) -> int {
    CycleGraph& cg = f->cg;
    int e;
    if (!graph_fresh() && (e = capture_cycle())) return e;
    for (int64_t c = 0; c < R; ++c) {
      // the inner target as in the host loop: max(t_abs, t_rel beta)
      if (mixed) {
        prm_h[c] = rtol * bnorm[c] * tscale[c];
        prm_h[R + c] = 2e-7;
      } else {
        prm_h[c] = 0.0;
        prm_h[R + c] = rtol * tscale[c] / std::max(res_r[c] * bnorm[c], 1e-300) * bnorm[c];
      }
      prm_h[2 * R + c] = bnorm[c];
      prm_h[3 * R + c] = done[c] ? 1.0 : 0.0;
    }
    const int ctl_in[2] = {std::min(m, maxit - iters), 0};
    int ctl_out[2] = {0, 0};
    cudaMemcpyAsync((void*)cyc.prm, prm_h.data(), prm_h.size() * sizeof(double), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(cyc.ctl, ctl_in, sizeof(ctl_in), cudaMemcpyHostToDevice, st);
    if (cudaGraphLaunch(cg.exec, st) != cudaSuccess) { set_error("hb_gmres: graph launch failed"); return HB_ECUDA; }
    ++graph_launches;
    int herr = 0;
    GridBar* gbar = (GridBar*)df.bar;
    cudaMemcpyAsync(ctl_out, cyc.ctl, sizeof(ctl_out), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(kuse_h.data(), cyc.kuse, R * sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(pres_h.data(), cyc.pres, R * sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(&herr, &gbar->err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("hb_gmres: CUDA error in the graph"); return HB_ECUDA; }
    if (herr) {
      cudaMemsetAsync(&gbar->err, 0, sizeof(int), st);
      set_error("a bounded device-side wait expired in a sweep kernel during the solve");
      return HB_ETIMEOUT;
    }
    if ((e = f->prof.harvest(ctl_out[1]))) { set_error("hb_gmres: reading the graph's timing events failed"); return e; }
    kcyc = ctl_out[1];
    iters += kcyc;
    for (int64_t c = 0; c < R; ++c) {
      if (done[c]) continue;
      it_r[c] += kuse_h[c] < 0 ? -kuse_h[c] : kcyc;
      pres_r[c] = pres_h[c];
    }
    return HB_OK;
  };

  // a capture that the runtime refuses leaves this call to the host-driven loop
  // (info->graph_launches stays 0)
  if (use_graph && !graph_fresh() && capture_cycle() != HB_OK) use_graph = false;

  while (iters < maxit) {
    nconv = 0;
    bool bad = false;
    for (int64_t c = 0; c < R; ++c) { done[c] = res_r[c] <= rtol; nconv += done[c]; bad |= !std::isfinite(res_r[c]); }
    if (nconv == R || bad) break;   // a non-finite residual ends the solve (reported as HB_ENAN)
    int kcyc = 0;
    const void* cdev = d.red_out;   // the cycle's combination coefficients (device)
    if (use_graph) {
      if ((rc = graph_cycle(kcyc))) return rc;
      cdev = coefd;
    } else {
      // ---- start vector
      std::vector<double> beta;
      if (!mixed) {
        if ((rc = sweep_internal(f, PREC_F64, lo, r, R, st))) return rc;   // r <- L'^{-1} r
      }
      if ((rc = norms(d, r, beta))) return rc;
      if (mixed) normalise(d, r, beta, V32);
      else normalise(d, r, beta, V);
      std::vector<double> target(R);
      for (int64_t c = 0; c < R; ++c) {
        gv[c].reset(m, beta[c]);
        kuse[c] = 0;
        // aim the inner estimate at the final tolerance (scaled back when the true residual missed)
        double want = rtol * bnorm[c] * tscale[c];
        if (mixed) want = std::max(want, 2e-7 * beta[c]);
        else want = rtol * tscale[c] * beta[c] / std::max(res_r[c] * bnorm[c], 1e-300) * bnorm[c];
        target[c] = want;
      }
      int j = 0;
      for (; j < m && iters < maxit; ++j) {
        double2* vj = mixed ? nullptr : V + (size_t)j * n * R;
        double2* w = mixed ? nullptr : V + (size_t)(j + 1) * n * R;
        if (!mixed) {
          // w = L'^{-1} A U'^{-1} v_j
          cudaMemcpyAsync(w, vj, vbytes, cudaMemcpyDeviceToDevice, st);
          if ((rc = sweep_internal(f, PREC_F64, up, w, R, st))) return rc;
          if ((rc = apply_internal(f, PREC_F64, adj, w, tmp2, R, st))) return rc;
          cudaMemcpyAsync(w, tmp2, vbytes, cudaMemcpyDeviceToDevice, st);
          if ((rc = sweep_internal(f, PREC_F64, lo, w, R, st))) return rc;
        } else {
          // z_j = M^{-1} v_j, w = A z_j, all in complex FP32
          float2* zj = zf + (size_t)j * n * R;
          float2* w32 = V32 + (size_t)(j + 1) * n * R;
          cudaMemcpyAsync(zj, V32 + (size_t)j * n * R, (size_t)n * R * sizeof(float2), cudaMemcpyDeviceToDevice, st);
          if ((rc = sweep_internal(f, PREC_F32, lo, zj, R, st))) return rc;
          if ((rc = sweep_internal(f, PREC_F32, up, zj, R, st))) return rc;
          if ((rc = apply_internal(f, PREC_F32, adj, zj, w32, R, st))) return rc;
        }
        if (mixed) {
          float2* w32 = V32 + (size_t)(j + 1) * n * R;
          if ((rc = cgs2(d, V32, (int64_t)n * R, j + 1, w32, h, hn))) return rc;
          normalise(d, w32, hn, w32);
        } else {
          if ((rc = cgs2(d, V, (int64_t)n * R, j + 1, w, h, hn))) return rc;
          normalise(d, w, hn, w);
        }
        ++iters;
        int active = 0;
        for (int64_t c = 0; c < R; ++c) {
          if (done[c] || kuse[c] < 0) continue;
          std::vector<zc> col(j + 1);
          for (int i = 0; i <= j; ++i) col[i] = h[(size_t)i * R + c];
          double est = gv[c].push(j, col.data(), hn[c]);
          pres_r[c] = bnorm[c] > 0 ? est / bnorm[c] : 0.0;
          it_r[c]++;
          if (est <= target[c]) kuse[c] = -(j + 1);   // converged in this cycle after j+1 steps
          else active++;
        }
        if (active == 0) { ++j; break; }
      }
      // ---- update the iterate with each column's own step count
      kcyc = j;
      std::fill(coef.begin(), coef.end(), zc(0.0));
      for (int64_t c = 0; c < R; ++c) {
        if (done[c]) continue;
        int k = kuse[c] < 0 ? -kuse[c] : kcyc;
        std::vector<zc> cf(k);
        gv[c].solve(k, cf.data());
        for (int i = 0; i < k; ++i) coef[(size_t)i * R + c] = cf[i];
      }
      std::vector<float2> coef32;
      if (mixed) {
        coef32.resize((size_t)kcyc * R);
        for (size_t i = 0; i < coef32.size(); ++i) coef32[i] = float2{(float)coef[i].real(), (float)coef[i].imag()};
        cudaMemcpyAsync(d.red_out, coef32.data(), coef32.size() * sizeof(float2), cudaMemcpyHostToDevice, st);
      } else {
        cudaMemcpyAsync(d.red_out, coef.data(), (size_t)kcyc * R * sizeof(double2), cudaMemcpyHostToDevice, st);
      }
    }
    if (!mixed) {
      // y += V c;  x = U'^{-1} y is formed for the residual check
      k_add_combo<double2><<<gsz(n * R), 256, 0, st>>>(V, (int64_t)n * R, kcyc, (const double2*)cdev, xv, n, R); count_launch(f, 1);
      cudaMemcpyAsync(tmp2, xv, vbytes, cudaMemcpyDeviceToDevice, st);
      double2* xs = tmp2;
      if ((rc = sweep_internal(f, PREC_F64, up, xs, R, st))) return rc;
      // r = b^ - A^ x (uses tmp2 as scratch: keep x in r first)
      cudaMemcpyAsync(r, xs, vbytes, cudaMemcpyDeviceToDevice, st);
      if ((rc = apply_internal(f, PREC_F64, adj, r, tmp2, R, st))) return rc;
      k_sub_into<<<gsz(n * R), 256, 0, st>>>(bh, tmp2, r, n * R); count_launch(f, 1);
      std::vector<double> rn;
      if ((rc = norms(d, r, rn))) return rc;
      for (int64_t c = 0; c < R; ++c) {
        double nr = bnorm[c] > 0 ? rn[c] / bnorm[c] : 0.0;
        if (!done[c] && nr > rtol) tscale[c] *= std::min(0.5, rtol / nr);
        res_r[c] = nr;
      }
    } else {
      // x += Z c  (Z in FP32), then the residual.  While some column's
      // residual is still large the whole residual is recomputed with FP64
      // arithmetic (its rounding must stay far below rtol relative to
      // ||A|| ||x||).  Once every column is within 1e-3, the correction dz = Z c
      // is small and r -= A dz is formed with the FP32 apply and accumulated
      // in FP64: its rounding is ~1e-7 of ||A dz|| <= 1e-3 ||b||.
      double worst_prev = 0.0;
      for (int64_t c = 0; c < R; ++c) worst_prev = std::max(worst_prev, res_r[c]);
      if (worst_prev > 1e-3) {
        k_add_combo<float2><<<gsz(n * R), 256, 0, st>>>(zf, (int64_t)n * R, kcyc, (const float2*)cdev, xv, n, R); count_launch(f, 1);
        if ((rc = true_residual(xv, r))) return rc;
      } else {
        cudaMemsetAsync(tmp2, 0, vbytes, st);   // dz in FP64, then rounded once to FP32
        k_add_combo<float2><<<gsz(n * R), 256, 0, st>>>(zf, (int64_t)n * R, kcyc, (const float2*)cdev, tmp2, n, R); count_launch(f, 1);
        k_axpy1<double2><<<gsz(n * R), 256, 0, st>>>(tmp2, xv, n * R); count_launch(f, 1);
        k_to_f32<<<gsz(n * R), 256, 0, st>>>(tmp2, f32s, n * R); count_launch(f, 1);
        float2* adz = (float2*)tmp2;   // A dz (FP32) reuses the scratch
        if ((rc = apply_internal(f, PREC_F32, adj, f32s, adz, R, st))) return rc;
        k_sub_f32<<<gsz(n * R), 256, 0, st>>>(adz, r, n * R); count_launch(f, 1);
        std::vector<double> rn;
        if ((rc = norms(d, r, rn))) return rc;
        for (int64_t c = 0; c < R; ++c) res_r[c] = bnorm[c] > 0 ? rn[c] / bnorm[c] : 0.0;
      }
    }
    ++cycles;
  }
  // final solution in the caller's layout (physical x: unaffected by the rescaling)
  if (!mixed) {
    cudaMemcpyAsync(tmp2, xv, vbytes, cudaMemcpyDeviceToDevice, st);
    if ((rc = sweep_internal(f, PREC_F64, up, tmp2, R, st))) return rc;
    if ((rc = launch_scatter_cols(tmp2, 0, n, R, x, 0, ld, 1.0, st))) return rc;
  } else {
    if ((rc = launch_scatter_cols(xv, 0, n, R, x, 0, ld, 1.0, st))) return rc;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("hb_gmres: CUDA error"); return HB_ECUDA; }
  if ((rc = hb_status(f, stream))) return rc;   // the last sweep's bounded waits
  nconv = 0;
  double worst = 0.0, worst_p = 0.0;
  bool nonfinite = false;
  for (int64_t c = 0; c < R; ++c) {
    nconv += res_r[c] <= rtol;
    nonfinite |= !std::isfinite(res_r[c]);
    worst = nan_max(worst, res_r[c]);
    worst_p = nan_max(worst_p, pres_r[c]);
  }
  if (info) {
    int32_t* ipr = info->iters_per_rhs;
    double* rpr = info->res_per_rhs;
    info->iters = iters;
    info->restarts = cycles;
    info->ir_steps = mixed ? cycles : 0;
    info->converged = nconv;
    info->true_rel_res = worst;
    info->precond_rel_res = worst_p;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (ipr) for (int64_t c = 0; c < R; ++c) ipr[c] = it_r[c];
    info->graph_launches = graph_launches;
    if (rpr) for (int64_t c = 0; c < R; ++c) rpr[c] = res_r[c];
  }
  if (nonfinite) {
    set_error("hb_gmres: the residual became non-finite after %d iterations (overflow in the preconditioned "
              "iteration)", iters);
    return HB_ENAN;
  }
  if (nconv < R) { set_error("hb_gmres: %d of %lld columns did not reach rtol in %d iterations", (int)(R - nconv), (long long)R, iters); return HB_ENOCONV; }
  return HB_OK;
}

// ---------------------------------------------------------------------------
// TFQMR (the solver of Sec. 4): Freund's transpose-free QMR on the split system
// L'^{-1} A U'^{-1} y = L'^{-1} b, x = U'^{-1} y, FP64 vectors, right-hand sides in
// lockstep with per-column scalars.  Half step m (even: a new alpha = rho /
// <r*, v> and the first direction u; odd: the second direction u - alpha v)
// updates the squared residual w, the QMR direction d and the iterate (theta,
// c, tau, eta); after an odd step rho' = <r*, w>, beta = rho' / rho,
// u = w + beta u_2 and v = A u + beta (A u_2 + beta v).  tau sqrt(m + 1)
// bounds the split residual; when it reaches rtol ||L'^{-1} b|| the true
// residual is formed and the bound tightened if it misses.  Columns that have
// converged (or broken down) get zero coefficients and stay frozen.
// ---------------------------------------------------------------------------
extern "C" int hb_tfqmr(hb_factor_t f, int op, const void* b_phys, const void* rstar, void* x, int64_t nrhs,
                        int64_t ld, double rtol, int maxit, hb_gmres_info* info, void* stream) {
  int rc = check_vec_args(f, b_phys, x, nrhs, ld, "hb_tfqmr");
  if (rc) return rc;
  if (op != HB_OP_N && op != HB_OP_H) { set_error("hb_tfqmr: bad op"); return HB_EINVAL; }
  if (!(rtol > 0) || maxit < 1) { set_error("hb_tfqmr: bad rtol/maxit"); return HB_EINVAL; }
  if (rstar == x) { set_error("hb_tfqmr: rstar and x must not alias"); return HB_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  auto t0 = std::chrono::steady_clock::now();
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("hb_tfqmr: stream error"); return HB_ECUDA; }
  const DevFactor& df = f->df;
  // operator arithmetic: FP64 for HB_C128; FP64 arithmetic on the complex-FP32
  // factors otherwise (the vectors and the iteration stay FP64 in every form)
  const Prec px = df.form == HB_C128 ? PREC_F64 : PREC_F32_ACC64;
  const int64_t n = df.n, R = nrhs, nR = n * R;
  const bool adj = op == HB_OP_H;
  const int lo = adj ? 3 : 0, up = adj ? 2 : 1;
  const size_t vbytes = (size_t)nR * sizeof(double2);
  Workspace& ws = f->ws;
  double2* bh = (double2*)ws.get(WS_VEC2, vbytes);
  double2* y = (double2*)ws.get(WS_VEC3, vbytes);
  double2* t1 = (double2*)ws.get(WS_VEC0, vbytes);
  double2* t2 = (double2*)ws.get(WS_VEC1, vbytes);
  double2* blk = (double2*)ws.get(WS_BASIS, vbytes * 8);
  double2* red = (double2*)ws.get(WS_RED, ((size_t)kRedBlocks * R + 6 * (size_t)R) * sizeof(double2));
  int* flag = (int*)ws.get(WS_SMALL, 256);
  if (!bh || !y || !t1 || !t2 || !blk || !red || !flag) { set_error("hb_tfqmr: workspace allocation failed"); return HB_ENOMEM; }
  double2 *w = blk, *u = blk + nR, *v = blk + 2 * nR, *au = blk + 3 * nR, *dd = blk + 4 * nR, *rs = blk + 5 * nR,
          *u2 = blk + 6 * nR, *rr = blk + 7 * nR;
  Dev d{f, st, n, R, red, red + (size_t)kRedBlocks * R, (double*)(red + (size_t)kRedBlocks * R + R)};
  double2* coef = red + (size_t)kRedBlocks * R + 2 * R;   // 4 x R per-column coefficients

  // non-finite inputs
  cudaMemsetAsync(flag, 0, sizeof(int), st);
  k_nonfinite<<<gsz(nR), 256, 0, st>>>((const double2*)b_phys, ld, n, R, flag); count_launch(f, 1);
  if (rstar) { k_nonfinite<<<gsz(nR), 256, 0, st>>>((const double2*)rstar, ld, n, R, flag); count_launch(f, 1); }
  int hflag = 0;
  cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("hb_tfqmr: CUDA error"); return HB_ECUDA; }
  if (hflag) { set_error("hb_tfqmr: b or rstar contains NaN/Inf"); return HB_ENAN; }

  // w = u = L'^{-1} b^,  r* (caller's, else w),  y = d = 0,  v = A u
  auto opf = [&](const double2* z, double2* out) -> int {   // out = L'^{-1} A U'^{-1} z
    int e;
    cudaMemcpyAsync(t1, z, vbytes, cudaMemcpyDeviceToDevice, st);
    if ((e = sweep_internal(f, px, up, t1, R, st))) return e;
    if ((e = apply_internal(f, px, adj, t1, out, R, st))) return e;
    return sweep_internal(f, px, lo, out, R, st);
  };
  auto upload = [&](const std::vector<zc>& c, int slot) -> double2* {
    double2* dst = coef + (size_t)slot * R;
    cudaMemcpyAsync(dst, c.data(), R * sizeof(double2), cudaMemcpyHostToDevice, st);
    return dst;
  };
  if ((rc = launch_gather_cols(b_phys, 0, ld, n, R, bh, 0, df.scale, st))) return rc;
  std::vector<double> bnorm, tau;
  if ((rc = norms(d, bh, bnorm))) return rc;
  cudaMemcpyAsync(w, bh, vbytes, cudaMemcpyDeviceToDevice, st);
  if ((rc = sweep_internal(f, px, lo, w, R, st))) return rc;
  cudaMemcpyAsync(u, w, vbytes, cudaMemcpyDeviceToDevice, st);
  if (rstar) { if ((rc = launch_gather_cols(rstar, 0, ld, n, R, rs, 0, 1.0, st))) return rc; }
  else cudaMemcpyAsync(rs, w, vbytes, cudaMemcpyDeviceToDevice, st);
  cudaMemsetAsync(y, 0, vbytes, st);
  cudaMemsetAsync(dd, 0, vbytes, st);
  if ((rc = opf(u, v))) return rc;
  cudaMemcpyAsync(au, v, vbytes, cudaMemcpyDeviceToDevice, st);
  if ((rc = norms(d, w, tau))) return rc;
  std::vector<zc> rho, alpha(R, zc(0.0)), eta(R, zc(0.0)), cz(R);
  if ((rc = dots(d, rs, 0, 1, w, rho))) return rc;
  std::vector<double> theta(R, 0.0), target(R), res_r(R, 1.0), bound(R, 1.0), tau0(tau), rn;
  std::vector<char> active(R, 1), broken(R, 0);
  std::vector<int32_t> it_r(R, 0);
  for (int64_t c = 0; c < R; ++c) {
    target[c] = rtol * tau[c];
    if (!(bnorm[c] > 0)) { active[c] = 0; res_r[c] = 0.0; bound[c] = 0.0; }
  }
  auto true_residual = [&]() -> int {   // res_r = ||b^ - A U'^{-1} y|| / ||b^||
    int e;
    cudaMemcpyAsync(t2, y, vbytes, cudaMemcpyDeviceToDevice, st);
    if ((e = sweep_internal(f, px, up, t2, R, st))) return e;
    if ((e = apply_internal(f, px, adj, t2, t1, R, st))) return e;
    k_sub_into<<<gsz(nR), 256, 0, st>>>(bh, t1, rr, nR); count_launch(f, 1);
    if ((e = norms(d, rr, rn))) return e;
    for (int64_t c = 0; c < R; ++c) res_r[c] = bnorm[c] > 0 ? rn[c] / bnorm[c] : 0.0;
    return HB_OK;
  };
  auto n_active = [&]() { int k = 0; for (int64_t c = 0; c < R; ++c) k += active[c]; return k; };
  int m = 0, checks = 0;
  while (m < maxit && n_active() > 0) {
    const bool even = (m % 2) == 0;
    double2* cur = u;
    if (even) {
      std::vector<zc> sig;
      if ((rc = dots(d, rs, 0, 1, v, sig))) return rc;
      for (int64_t c = 0; c < R; ++c) {
        if (!active[c]) { alpha[c] = 0.0; continue; }
        if (!(std::abs(sig[c]) > 0) || !std::isfinite(std::abs(sig[c])) || !(std::abs(rho[c]) > 0)) {
          active[c] = 0; broken[c] = 1; alpha[c] = 0.0; continue;   // Lanczos breakdown
        }
        alpha[c] = rho[c] / sig[c];
      }
      cudaMemcpyAsync(u2, u, vbytes, cudaMemcpyDeviceToDevice, st);      // u2 = u - alpha v
      k_sub_combo<double2><<<gsz(nR), 256, 0, st>>>(v, 0, 1, upload(alpha, 0), u2, n, R); count_launch(f, 1);
    } else {
      cur = u2;
      if ((rc = opf(u2, au))) return rc;                                  // au = A u2
    }
    for (int64_t c = 0; c < R; ++c) cz[c] = active[c] ? alpha[c] : zc(0.0);
    k_sub_combo<double2><<<gsz(nR), 256, 0, st>>>(au, 0, 1, upload(cz, 1), w, n, R); count_launch(f, 1);   // w -= alpha A cur
    for (int64_t c = 0; c < R; ++c) cz[c] = active[c] ? theta[c] * theta[c] * eta[c] / alpha[c] : zc(0.0);
    k_xpay<<<gsz(nR), 256, 0, st>>>(cur, upload(cz, 2), dd, n, R); count_launch(f, 1);                      // d = cur + s d
    std::vector<double> wn;
    if ((rc = norms(d, w, wn))) return rc;
    for (int64_t c = 0; c < R; ++c) {
      if (!active[c]) { cz[c] = 0.0; continue; }
      theta[c] = wn[c] / tau[c];
      const double cc = 1.0 / std::sqrt(1.0 + theta[c] * theta[c]);
      tau[c] *= theta[c] * cc;
      eta[c] = cc * cc * alpha[c];
      cz[c] = eta[c];
    }
    k_add_combo<double2><<<gsz(nR), 256, 0, st>>>(dd, 0, 1, upload(cz, 3), y, n, R); count_launch(f, 1);   // y += eta d
    if (!even) {
      std::vector<zc> rho_new, beta(R, zc(0.0));
      if ((rc = dots(d, rs, 0, 1, w, rho_new))) return rc;
      for (int64_t c = 0; c < R; ++c) {
        if (!active[c]) continue;
        beta[c] = rho_new[c] / rho[c];   // rho != 0: checked when alpha was formed
        rho[c] = rho_new[c];
      }
      double2* bz = upload(beta, 0);
      k_xpay<<<gsz(nR), 256, 0, st>>>(w, bz, u2, n, R); count_launch(f, 1);    // u2 = w + beta u2: the new u
      std::swap(u, u2);
      k_xpay<<<gsz(nR), 256, 0, st>>>(au, bz, v, n, R); count_launch(f, 1);    // v = A u2_old + beta v
      if ((rc = opf(u, au))) return rc;                                         // au = A u
      k_xpay<<<gsz(nR), 256, 0, st>>>(au, bz, v, n, R); count_launch(f, 1);    // v = A u + beta v
    }
    ++m;
    bool check = false;
    for (int64_t c = 0; c < R; ++c) {
      if (!active[c]) continue;
      it_r[c] = m;
      bound[c] = tau[c] * std::sqrt(m + 1.0) / tau0[c];
      if (tau[c] * std::sqrt(m + 1.0) <= target[c]) check = true;
    }
    if (check) {
      if ((rc = true_residual())) return rc;
      ++checks;
      for (int64_t c = 0; c < R; ++c) {
        if (!active[c]) continue;
        if (res_r[c] <= rtol) active[c] = 0;
        else if (!(tau[c] > 0)) { active[c] = 0; broken[c] = 1; }   // w = 0 but x misses rtol
        else if (tau[c] * std::sqrt(m + 1.0) <= target[c]) target[c] *= std::min(0.5, rtol / res_r[c]);
      }
    }
  }
  // report the final true residual of every column, return x = U'^{-1} y
  if ((rc = true_residual())) return rc;
  if ((rc = launch_scatter_cols(t2, 0, n, R, x, 0, ld, 1.0, st))) return rc;
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("hb_tfqmr: CUDA error"); return HB_ECUDA; }
  if ((rc = hb_status(f, stream))) return rc;   // the last sweep's bounded waits
  int nconv = 0, nbroken = 0;
  double worst = 0.0, worst_b = 0.0;
  for (int64_t c = 0; c < R; ++c) {
    nconv += res_r[c] <= rtol;
    nbroken += broken[c];
    worst = nan_max(worst, res_r[c]);
    worst_b = nan_max(worst_b, bound[c]);
  }
  if (info) {
    info->iters = m;
    info->restarts = checks;
    info->ir_steps = 0;
    info->converged = nconv;
    info->true_rel_res = worst;
    info->precond_rel_res = worst_b;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    info->graph_launches = 0;
    if (info->iters_per_rhs) for (int64_t c = 0; c < R; ++c) info->iters_per_rhs[c] = it_r[c];
    if (info->res_per_rhs) for (int64_t c = 0; c < R; ++c) info->res_per_rhs[c] = res_r[c];
  }
  if (std::isnan(worst)) {
    set_error("hb_tfqmr: the residual became non-finite after %d half steps", m);
    return HB_ENAN;
  }
  if (nconv < R) {
    set_error("hb_tfqmr: %d of %lld columns did not reach rtol in %d half steps (%d broke down)", (int)(R - nconv),
              (long long)R, m, nbroken);
    return HB_ENOCONV;
  }
  return HB_OK;
}

extern "C" int hb_rhs_plane_wave(hb_factor_t f, const double* phi_deg, int64_t nrhs, void* b, int64_t ld, void* stream) {
  if (!f || !phi_deg || !b || nrhs < 1 || ld < f->df.n) { set_error("hb_rhs_plane_wave: bad argument"); return HB_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> cs(2 * nrhs);
  for (int64_t r = 0; r < nrhs; ++r) {
    double ph = phi_deg[r] * M_PI / 180.0;
    cs[r] = std::cos(ph);
    cs[nrhs + r] = std::sin(ph);
  }
  double* d = (double*)f->ws.get(WS_SMALL, std::max<size_t>(256, cs.size() * sizeof(double)));
  if (!d) { set_error("hb_rhs_plane_wave: allocation failed"); return HB_ENOMEM; }
  cudaMemcpyAsync(d, cs.data(), cs.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  k_plane_wave<<<gsz(f->df.n * nrhs), 256, 0, st>>>(f->df.cx, f->df.cy, f->df.n, d, d + nrhs, nrhs, f->df.kappa,
                                                    (double2*)b, ld); count_launch(f, 1);
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("hb_rhs_plane_wave: CUDA error"); return HB_ECUDA; }
  return HB_OK;
}

static int far_common(hb_factor_t f, const void* x, int64_t nrhs, int64_t ld, const double* phi, int64_t nang,
                      void* out, void* stream, bool mono) {
  if (!f || !x || !phi || !out || nrhs < 1 || ld < f->df.n || nang < 1) { set_error("hb_far_field: bad argument"); return HB_EINVAL; }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> cs(2 * nang);
  for (int64_t q = 0; q < nang; ++q) {
    double ph = phi[q] * M_PI / 180.0;
    cs[q] = std::cos(ph);
    cs[nang + q] = std::sin(ph);
  }
  double* d = (double*)f->ws.get(WS_SMALL, std::max<size_t>(256, cs.size() * sizeof(double)));
  if (!d) { set_error("hb_far_field: allocation failed"); return HB_ENOMEM; }
  cudaMemcpyAsync(d, cs.data(), cs.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  const double k = f->df.kappa;
  // C = -(k eta0 / 4) sqrt(2i / (pi k))
  std::complex<double> C = -(k * f->df.eta0 / 4.0) * std::sqrt(std::complex<double>(0.0, 2.0 / (M_PI * k)));
  dim3 grid((unsigned)(mono ? 1 : nang), (unsigned)nrhs);
  k_far_field<<<grid, 256, 0, st>>>(f->df.cx, f->df.cy, f->df.w, f->df.n, (const double2*)x, ld, d, d + nang, nang, k,
                                    double2{C.real(), C.imag()}, (double2*)out, mono ? 1 : 0); count_launch(f, 1);
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("hb_far_field: CUDA error"); return HB_ECUDA; }
  return HB_OK;
}

extern "C" int hb_far_field(hb_factor_t f, const void* x, int64_t nrhs, int64_t ld, const double* phi_obs_deg,
                            int64_t nobs, void* out, void* stream) {
  return far_common(f, x, nrhs, ld, phi_obs_deg, nobs, out, stream, false);
}

extern "C" int hb_far_field_adjoint(hb_factor_t f, const void* g, int64_t nrhs, const double* phi_obs_deg,
                                    int64_t nobs, void* out, int64_t ld, void* stream) {
  if (!f || f->host_only || !g || !phi_obs_deg || !out || nrhs < 1 || nobs < 1 || ld < f->df.n) {
    set_error("hb_far_field_adjoint: bad argument");
    return HB_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<double> cs(2 * nobs);
  for (int64_t q = 0; q < nobs; ++q) {
    double ph = phi_obs_deg[q] * M_PI / 180.0;
    cs[q] = std::cos(ph);
    cs[nobs + q] = std::sin(ph);
  }
  double* d = (double*)f->ws.get(WS_SMALL, std::max<size_t>(256, cs.size() * sizeof(double)));
  if (!d) { set_error("hb_far_field_adjoint: allocation failed"); return HB_ENOMEM; }
  cudaMemcpyAsync(d, cs.data(), cs.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  const double k = f->df.kappa;
  std::complex<double> C = -(k * f->df.eta0 / 4.0) * std::sqrt(std::complex<double>(0.0, 2.0 / (M_PI * k)));
  std::complex<double> Cc = std::conj(C);
  k_far_field_adj<<<gsz(f->df.n * nrhs), 256, 0, st>>>(f->df.cx, f->df.cy, f->df.w, f->df.n, (const double2*)g, nobs,
                                                       d, d + nobs, nrhs, k, double2{Cc.real(), Cc.imag()},
                                                       (double2*)out, ld);
  count_launch(f, 1);
  if (cudaStreamSynchronize(st) != cudaSuccess) { set_error("hb_far_field_adjoint: CUDA error"); return HB_ECUDA; }
  return HB_OK;
}

extern "C" int hb_monostatic(hb_factor_t f, const void* x, int64_t nrhs, int64_t ld, const double* phi_deg, void* out,
                             void* stream) {
  return far_common(f, x, nrhs, ld, phi_deg, nrhs, out, stream, true);
}
