// libftgcr: C ABI, setup kernels and launch logic of the GB300-native FT-GCR(k)
// solver (Gillard & Benacchio, arXiv 2103.07210, Algorithm 1).  See
// include/ftgcr.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <type_traits>
#include <vector>

#include "../../include/ftgcr.h"
#include "ftgcr_device.cuh"
#include "ftgcr_phases.cuh"
#include "ftgcr_instances.h"
#include "ftgcr_serve.h"

using namespace ftgcr;

static_assert(sizeof(Fault) == sizeof(ftgcr_fault), "fault layout");
static_assert(sizeof(LossEv) == sizeof(ftgcr_loss), "loss layout");
static_assert(kMaxLosses == FTGCR_MAX_LOSSES, "max losses");
static_assert(kMaxK == FTGCR_MAX_K, "max k");
static_assert(kMaxFaults == FTGCR_MAX_FAULTS, "max faults");
static_assert(kMaxDetect == FTGCR_MAX_DETECT, "max detect");

namespace {

constexpr double kPi = 3.14159265358979323846;

// ------------------------------------------------------------ setup kernels
// Face coefficients of Eq. (1)'s finite-volume operator from the cell-centred
// coefficient D and the per-row geometry; same expressions, in the same
// order, as the definition (FP64, --fmad=false).
__global__ void k_face_coeffs(int nlon, int nlat, const double* __restrict__ D, const double* __restrict__ cx,
                              const double* __restrict__ cy, const double* __restrict__ area, double mu,
                              double* Tx, double* Ty, double* muA, float* Tx32, float* Ty32, float* muA32) {
  const long long N = (long long)nlon * nlat;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(g / nlon), i = (int)(g - (long long)j * nlon);
    const int ie = (i + 1) % nlon;
    const double tx = 0.5 * (D[g] + D[(long long)j * nlon + ie]) * cx[j];
    const double ty = (j == nlat - 1) ? 0.0 : 0.5 * (D[g] + D[g + nlon]) * cy[j];
    Tx[g] = tx;
    Ty[g] = ty;
    if (Tx32) {
      Tx32[g] = (float)tx;
      Ty32[g] = (float)ty;
    }
    if (i == 0) {
      const double m = mu * area[j];
      muA[j] = m;
      if (muA32) muA32[j] = (float)m;
    }
  }
}

// Line-preconditioner factorisation, one thread per latitude row (setup
// only).  Row system M x = b, M_ii = d_i = Tx_i + Tx_{i-1} + sigma_i,
// M_{i,i+1} = -Tx_i (periodic).  Thomas factorisation of the leading
// (n-1) x (n-1) block, operation for operation the CPU oracle's:
// w_0 = d_0, l_i = -Tx_{i-1} / w_{i-1}, w_i = d_i - l_i (-Tx_{i-1}),
// winv_i = 1 / w_i, u_i = -Tx_i winv_i; bordering vector z = A0^-1 c,
// c = (-Tx_{n-1}, 0, ..., 0, -Tx_{n-2}) by the same substitution; delta =
// d_{n-1} + Tx_{n-1} z_0 + Tx_{n-2} z_{n-2}.
// FP64 outputs (natural layout): l, winv, u, z, delta.  FP32 outputs (chunk
// layout, element i -> [row][i % C][i / C]): c = -u, winv, z, and per row
// 1/delta, Tx_{n-1}/delta, Tx_{n-2}/delta.  Jacobi: d_i (FP64) or 1/d_i (FP32).
__global__ void k_line_factor(int nlon, int nlat, int C, int precond, const double* __restrict__ Tx,
                              const double* __restrict__ Ty, const double* __restrict__ muA, double* l64,
                              double* w64, double* u64, double* z64, double* lrow64, float* lc32, float* lw32,
                              float* lz32, float* lrow32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nlat) return;
  const int n = nlon, m = n - 1;
  const long long rb = (long long)j * n;
  const double* tx = Tx + rb;
  auto diag = [&](int i) {
    const long long c = rb + i;
    double s = 0.0;
    if (j < nlat - 1) s = s + Ty[c];
    if (j > 0) s = s + Ty[c - n];
    s = s + muA[j];
    return tx[i] + tx[(i + n - 1) % n] + s;
  };
  if (precond == PC_JACOBI) {
    for (int i = 0; i < n; ++i) {
      const double d = diag(i);
      if (w64) w64[rb + i] = d;
      if (lw32) lw32[rb + i] = (float)(1.0 / d);
    }
    return;
  }
  if (precond != PC_LINE) return;
  double* l = l64 + rb;
  double* winv = w64 + rb;
  double* u = u64 + rb;
  double* z = z64 + rb;
  double w = diag(0);
  winv[0] = 1.0 / w;
  l[0] = 0.0;
  for (int i = 1; i < m; ++i) {
    l[i] = -tx[i - 1] / w;
    w = diag(i) - l[i] * -tx[i - 1];
    winv[i] = 1.0 / w;
  }
  for (int i = 0; i < m; ++i) u[i] = (i < m - 1) ? -tx[i] * winv[i] : 0.0;
  u[m] = 0.0;
  l[m] = 0.0;
  winv[m] = 0.0;
  // z = A0^-1 c
  for (int i = 0; i < m; ++i) z[i] = 0.0;
  z[0] = -tx[n - 1];
  z[m - 1] = z[m - 1] + -tx[n - 2];
  for (int i = 1; i < m; ++i) z[i] = fma(-l[i], z[i - 1], z[i]);
  z[m - 1] = z[m - 1] * winv[m - 1];
  for (int i = m - 2; i >= 0; --i) z[i] = fma(-u[i], z[i + 1], z[i] * winv[i]);
  z[m] = 0.0;
  const double delta = diag(n - 1) + tx[n - 1] * z[0] + tx[n - 2] * z[m - 1];
  lrow64[(long long)j * 4 + 0] = delta;
  lrow64[(long long)j * 4 + 1] = 0.0;
  lrow64[(long long)j * 4 + 2] = 0.0;
  lrow64[(long long)j * 4 + 3] = 0.0;
  if (lc32) {
    const long long cb = (long long)j * 32 * C;
    for (int i = 0; i < 32 * C; ++i) {
      const int lane = i / C, k = i % C;
      const long long pos = cb + (long long)k * 32 + lane;
      const bool in = i < m;
      lc32[pos] = in ? (float)(-u[i]) : 0.f;
      lw32[pos] = in ? (float)winv[i] : 0.f;
      lz32[pos] = in ? (float)z[i] : 0.f;
    }
    const double dinv = 1.0 / delta;
    lrow32[(long long)j * 4 + 0] = (float)dinv;
    lrow32[(long long)j * 4 + 1] = (float)(tx[n - 1] * dinv);
    lrow32[(long long)j * 4 + 2] = (float)(tx[n - 2] * dinv);
    lrow32[(long long)j * 4 + 3] = 0.f;
  }
}

// The same factorisation as k_line_factor, split into its three dependent
// chains and the elementwise work between them.  The chains run one lane per
// latitude row, 32 rows to a warp, because GB300's FP64 unit costs the same
// per warp instruction for 1 or 32 active lanes.  Each lane loads a block of
// inputs ahead while it steps through the current one.  The off-chain work
// runs one thread per element: the diagonal, the reciprocal pivots, u, the
// products of the backward substitution and the FP32 layout.  Every value is
// formed by the same operations in the same order as in k_line_factor and the
// CPU oracle, so the factors are bitwise the same.
constexpr int kLfBlock = 8;  // inputs loaded ahead per lane

// d_i of every element (the diagonal of the row systems).
__global__ void k_lf_diag(int nlon, int nlat, const double* __restrict__ Tx, const double* __restrict__ Ty,
                          const double* __restrict__ muA, double* dg) {
  const long long N = (long long)nlon * nlat;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(g / nlon), i = (int)(g - (long long)j * nlon);
    double s = 0.0;
    if (j < nlat - 1) s = s + Ty[g];
    if (j > 0) s = s + Ty[g - nlon];
    s = s + muA[j];
    dg[g] = Tx[g] + Tx[(long long)j * nlon + (i + nlon - 1) % nlon] + s;
  }
}

// Chain 1: w_0 = d_0, l_i = -Tx_{i-1} / w_{i-1}, w_i = d_i - l_i (-Tx_{i-1}),
// i < m; l and the pivots w (not yet inverted) stored.
__global__ void k_lf_chain_lw(int nlon, int nlat, const double* __restrict__ Tx, const double* __restrict__ dg,
                              double* __restrict__ l, double* __restrict__ wout) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nlat) return;
  const int m = nlon - 1;
  const long long rb = (long long)j * nlon;
  const double* tx = Tx + rb;
  const double* d = dg + rb;
  double w = d[0];
  wout[rb] = w;
  l[rb] = 0.0;
  double ta[kLfBlock], da[kLfBlock], tb[kLfBlock], db[kLfBlock];
  auto load = [&](int i0, double* t, double* dd) {
#pragma unroll
    for (int q = 0; q < kLfBlock; ++q)
      if (i0 + q < m) {
        t[q] = tx[i0 + q - 1];
        dd[q] = d[i0 + q];
      }
  };
  auto step = [&](int i0, const double* t, const double* dd) {
#pragma unroll
    for (int q = 0; q < kLfBlock; ++q)
      if (i0 + q < m) {
        const double li = -t[q] / w;
        w = dd[q] - li * -t[q];
        l[rb + i0 + q] = li;
        wout[rb + i0 + q] = w;
      }
  };
  load(1, ta, da);
  for (int i0 = 1; i0 < m; i0 += 2 * kLfBlock) {
    load(i0 + kLfBlock, tb, db);
    step(i0, ta, da);
    load(i0 + 2 * kLfBlock, ta, da);
    step(i0 + kLfBlock, tb, db);
  }
}

// winv_i = 1 / w_i, u_i = -Tx_i winv_i (u_{m-1} = 0), the padding l_m = winv_m
// = u_m = 0, and the bordering right-hand side c into z:
// c = (-Tx_{n-1}, 0, ..., 0, 0 + -Tx_{n-2}), z_m = 0.
__global__ void k_lf_recip(int nlon, int nlat, const double* __restrict__ Tx, double* l, double* winv, double* u,
                           double* z) {
  const long long N = (long long)nlon * nlat;
  const int m = nlon - 1;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(g / nlon), i = (int)(g - (long long)j * nlon);
    const long long rb = (long long)j * nlon;
    if (i < m) {
      const double wi = 1.0 / winv[g];
      winv[g] = wi;
      u[g] = (i < m - 1) ? -Tx[g] * wi : 0.0;
      double c = 0.0;
      if (i == 0) c = -Tx[rb + nlon - 1];
      if (i == m - 1) c = c + -Tx[rb + nlon - 2];
      z[g] = c;
    } else {
      winv[g] = 0.0;
      u[g] = 0.0;
      l[g] = 0.0;
      z[g] = 0.0;
    }
  }
}

// Chain 2: forward substitution of c, z_i = fma(-l_i, z_{i-1}, z_i), i < m.
__global__ void k_lf_chain_fwd(int nlon, int nlat, const double* __restrict__ l, double* __restrict__ z) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nlat) return;
  const int m = nlon - 1;
  const long long rb = (long long)j * nlon;
  double y = z[rb];
  double la[kLfBlock], ca[kLfBlock], lb[kLfBlock], cb[kLfBlock];
  auto load = [&](int i0, double* ll, double* cc) {
#pragma unroll
    for (int q = 0; q < kLfBlock; ++q)
      if (i0 + q < m) {
        ll[q] = l[rb + i0 + q];
        cc[q] = z[rb + i0 + q];
      }
  };
  auto step = [&](int i0, const double* ll, const double* cc) {
#pragma unroll
    for (int q = 0; q < kLfBlock; ++q)
      if (i0 + q < m) {
        y = fma(-ll[q], y, cc[q]);
        z[rb + i0 + q] = y;
      }
  };
  load(1, la, ca);
  for (int i0 = 1; i0 < m; i0 += 2 * kLfBlock) {
    load(i0 + kLfBlock, lb, cb);
    step(i0, la, ca);
    load(i0 + 2 * kLfBlock, la, ca);
    step(i0 + kLfBlock, lb, cb);
  }
}

// The backward step's products z_i winv_i, i < m (z_{m-1} winv_{m-1} is also
// the first value of the backward substitution).
__global__ void k_lf_products(int nlon, int nlat, const double* __restrict__ winv, double* z) {
  const long long N = (long long)nlon * nlat;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(g % nlon);
    if (i < nlon - 1) z[g] = z[g] * winv[g];
  }
}

// Chain 3: backward substitution z_i = fma(-u_i, z_{i+1}, z_i winv_i),
// i = m-2 .. 0, then delta = d_{n-1} + Tx_{n-1} z_0 + Tx_{n-2} z_{m-1} and the
// row constants (FP64: delta, then 1/delta, Tx_{n-1}/delta, Tx_{n-2}/delta;
// FP32: the last three).
__global__ void k_lf_chain_bwd(int nlon, int nlat, const double* __restrict__ Tx, const double* __restrict__ Ty,
                               const double* __restrict__ muA, const double* __restrict__ u, double* __restrict__ z,
                               double* lrow64, float* lrow32) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nlat) return;
  const int n = nlon, m = n - 1;
  const long long rb = (long long)j * n;
  double y = z[rb + m - 1];
  double ua[kLfBlock], pa[kLfBlock], ub[kLfBlock], pb[kLfBlock];
  auto load = [&](int i1, double* uu, double* pp) {  // elements i1, i1 - 1, ...
#pragma unroll
    for (int q = 0; q < kLfBlock; ++q)
      if (i1 - q >= 0) {
        uu[q] = u[rb + i1 - q];
        pp[q] = z[rb + i1 - q];
      }
  };
  auto step = [&](int i1, const double* uu, const double* pp) {
#pragma unroll
    for (int q = 0; q < kLfBlock; ++q)
      if (i1 - q >= 0) {
        y = fma(-uu[q], y, pp[q]);
        z[rb + i1 - q] = y;
      }
  };
  load(m - 2, ua, pa);
  for (int i1 = m - 2; i1 >= 0; i1 -= 2 * kLfBlock) {
    load(i1 - kLfBlock, ub, pb);
    step(i1, ua, pa);
    load(i1 - 2 * kLfBlock, ua, pa);
    step(i1 - kLfBlock, ub, pb);
  }
  const double* tx = Tx + rb;
  double s = 0.0;
  if (j < nlat - 1) s = s + Ty[rb + n - 1];
  if (j > 0) s = s + Ty[rb + n - 1 - n];
  s = s + muA[j];
  const double d_last = tx[n - 1] + tx[n - 2] + s;
  const double delta = d_last + tx[n - 1] * z[rb] + tx[n - 2] * z[rb + m - 1];
  const double dinv = 1.0 / delta;
  lrow64[(long long)j * 4 + 0] = delta;
  lrow64[(long long)j * 4 + 1] = dinv;
  lrow64[(long long)j * 4 + 2] = tx[n - 1] * dinv;
  lrow64[(long long)j * 4 + 3] = tx[n - 2] * dinv;
  if (lrow32) {
    lrow32[(long long)j * 4 + 0] = (float)dinv;
    lrow32[(long long)j * 4 + 1] = (float)(tx[n - 1] * dinv);
    lrow32[(long long)j * 4 + 2] = (float)(tx[n - 2] * dinv);
    lrow32[(long long)j * 4 + 3] = 0.f;
  }
}

// Constants in the per-lane chunk layout (FP32, or FP64 for the FP64 path's
// chunked row solve): position k*32 + lane of row j holds element
// i = lane*C + k (c = -u, winv, z; zero past the block).
template <typename O>
__global__ void k_lf_chunks(int nlon, int nlat, int C, const double* __restrict__ u, const double* __restrict__ winv,
                            const double* __restrict__ z, O* lc32, O* lw32, O* lz32) {
  const long long per = 32LL * C, total = per * nlat;
  const int m = nlon - 1;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(q / per);
    const int pos = (int)(q - (long long)j * per), k = pos >> 5, lane = pos & 31;
    const int i = lane * C + k;
    const bool in = i < m;
    const long long g = (long long)j * nlon + i;
    lc32[q] = in ? (O)(-u[g]) : O(0);
    lw32[q] = in ? (O)winv[g] : O(0);
    lz32[q] = in ? (O)z[g] : O(0);
  }
}

// FP32 constants in the piece-major layout of the streamed rounds: position
// L (C + 4) + kk of row j holds element i = L C + kk (c = -u, winv, z; zero
// past the leading block and in the padding).
__global__ void k_lf_pieces(int nlon, int nlat, int C, const double* __restrict__ u, const double* __restrict__ winv,
                            const double* __restrict__ z, float* lc, float* lw, float* lz) {
  const int P = C + 4;
  const long long per = 32LL * P, total = per * nlat;
  const int m = nlon - 1;
  for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total; q += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(q / per);
    const int pos = (int)(q - (long long)j * per), L = pos / P, kk = pos - L * P;
    const int i = L * C + kk;
    const bool in = kk < C && i < m;
    const long long g = (long long)j * nlon + i;
    lc[q] = in ? (float)(-u[g]) : 0.f;
    lw[q] = in ? (float)winv[g] : 0.f;
    lz[q] = in ? (float)z[g] : 0.f;
  }
}

// The line preconditioner's factorisation (Jacobi: its diagonal), enqueued
// on st.  FP64 outputs l, winv, u, z (z doubles as scratch for the diagonal)
// and the row constants; FP32 chunk-layout constants when lc32 is given.
int launch_line_factor(int nlon, int nlat, int C, int precond, const double* Tx, const double* Ty,
                       const double* muA, double* l64, double* w64, double* u64, double* z64, double* r64,
                       float* lc32, float* lw32, float* lz32, float* lrow32, cudaStream_t st, double* lcc = nullptr,
                       double* lwc = nullptr, double* lzc = nullptr, float* lcp = nullptr, float* lwp = nullptr,
                       float* lzp = nullptr) {
  if (precond != PC_LINE) {
    k_line_factor<<<(nlat + 63) / 64, 64, 0, st>>>(nlon, nlat, C, precond, Tx, Ty, muA, l64, w64, u64, z64, r64, lc32,
                                                   lw32, lz32, lrow32);
    return cudaGetLastError() == cudaSuccess ? FTGCR_OK : FTGCR_ERR_CUDA;
  }
  const long long N = (long long)nlon * nlat;
  const int eb = 256, eg = (int)std::min<long long>((N + eb - 1) / eb, 8192);
  const int rg = (nlat + 31) / 32;  // one lane per row, one warp per block
  k_lf_diag<<<eg, eb, 0, st>>>(nlon, nlat, Tx, Ty, muA, z64);
  k_lf_chain_lw<<<rg, 32, 0, st>>>(nlon, nlat, Tx, z64, l64, w64);
  k_lf_recip<<<eg, eb, 0, st>>>(nlon, nlat, Tx, l64, w64, u64, z64);
  k_lf_chain_fwd<<<rg, 32, 0, st>>>(nlon, nlat, l64, z64);
  k_lf_products<<<eg, eb, 0, st>>>(nlon, nlat, w64, z64);
  k_lf_chain_bwd<<<rg, 32, 0, st>>>(nlon, nlat, Tx, Ty, muA, u64, z64, r64, lrow32);
  const long long nc = 32LL * C * nlat;
  const int cgrid = (int)std::min<long long>((nc + eb - 1) / eb, 8192);
  if (lc32) k_lf_chunks<float><<<cgrid, eb, 0, st>>>(nlon, nlat, C, u64, w64, z64, lc32, lw32, lz32);
  if (lcc) k_lf_chunks<double><<<cgrid, eb, 0, st>>>(nlon, nlat, C, u64, w64, z64, lcc, lwc, lzc);
  if (lcp) {
    const long long np = 32LL * (C + 4) * nlat;
    k_lf_pieces<<<(int)std::min<long long>((np + eb - 1) / eb, 8192), eb, 0, st>>>(nlon, nlat, C, u64, w64, z64, lcp,
                                                                                 lwp, lzp);
  }
  return cudaGetLastError() == cudaSuccess ? FTGCR_OK : FTGCR_ERR_CUDA;
}

// out = L(in), FP64, one thread per element.
__global__ void k_apply_operator(const double* in, double* out, const double* Tx, const double* Ty, const double* muA,
                                 int nlon, int nlat) {
  const long long N = (long long)nlon * nlat;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(g / nlon), i = (int)(g - (long long)j * nlon);
    out[g] = stencil_global<double>(in, Tx, Ty, muA, nlon, nlat, j, i);
  }
}

// out = P^-1(in), FP64, one warp per latitude row (the solve of the
// persistent kernel's PA phase).
__global__ void k_apply_precond(const double* in, double* out, SolveDev<double> sd) {
  extern __shared__ __align__(16) unsigned char dsm[];
  double* sm = reinterpret_cast<double*>(dsm);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + warp;
  if (j >= sd.nlat) return;
  const int stride = row_stride(sd.nlon);
  double* row = sm + warp * stride;
  const long long base = (long long)j * sd.nlon;
  for (int i = lane; i < sd.nlon; i += 32) row[sk(i)] = in[base + i];
  __syncwarp();
  precond_row(sd, j, row, row_consts_global(sd, j));
  __syncwarp();
  for (int i = lane; i < sd.nlon; i += 32) out[base + i] = row[sk(i)];
}

// Per-solve start: record the call's pointers and fault plan in the device
// descriptor, reset the state machine and the launch control block.
struct BeginArgs {
  const double* R;
  const double* x0;
  double* xout;
  int nfaults;
  int nlosses;
  long long max_steps;
  Fault faults[kMaxFaults];
  LossEv losses[kMaxLosses];
};

// A batch launch's solve table (descriptor pointers and tile counts), filled
// from kernel parameters rather than a copy from host memory, so that a
// batch captured into a CUDA graph holds its own copy of the table.
constexpr int kTableChunk = 256;
struct BatchTable {
  void* sdev[kTableChunk];
  int nt[kTableChunk];
  int n, off;
};
__global__ void k_fill_table(BatchTable t, void** d_solves, int* d_nt) {
  const int i = threadIdx.x;
  if (i < t.n) {
    d_solves[t.off + i] = t.sdev[i];
    d_nt[t.off + i] = t.nt[i];
  }
}

// Flags a non-finite value of a staged input (exponent bits all ones).
__global__ void k_nonfinite(const double* __restrict__ a, long long n, LaunchCtl* ctl) {
  bool bad = false;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    bad |= ((__double_as_longlong(a[i]) >> 52) & 0x7FF) == 0x7FF;
  if (__syncthreads_or(bad) && threadIdx.x == 0) ctl->nonfinite = 1;
}

// check (host-array solves): the control block whose `nonfinite` flag
// k_nonfinite set over the staged inputs; a solve whose input is not finite
// records a finished, not-converged state and is not started.  ctl: the
// launch's control block to reset (single-solve and batch launches), or null.
template <typename T>
__global__ void k_begin_solve(SolveDev<T>* sd, BeginArgs b, int* active, int n_active, int slot, int par,
                              LaunchCtl* ctl, const LaunchCtl* check = nullptr) {
  if (check && check->nonfinite) {
    if (threadIdx.x == 0) {
      SolveState S;
      memset(&S, 0, sizeof S);
      S.status = ST_NOT_CONVERGED;
      S.refused = 1;
      *sd->result = S;
      active[slot] = 0;
      active[n_active + slot] = 0;
      if (ctl) {
        ctl->counter = 0;
        ctl->err = 0;
        ctl->round0 = 0;
        ctl->round_end = 0;
      }
    }
    return;
  }
  if (threadIdx.x == 0) {
    sd->R = b.R;
    sd->x0 = b.x0;
    sd->xout = b.xout;
    sd->nfaults = b.nfaults;
    sd->nlosses = b.nlosses;
    SolveState S;
    memset(&S, 0, sizeof S);
    S.active = 1;
    S.pending = K_NONE;
    S.first_out = 1;
    S.phiS = S.rS = 0;
    S.phiW = S.rW = 1;
    S.status = ST_RUNNING;
    // par < 0: the round parity of the launch that will run the solve is not
    // known yet (the solve joins a resumable launch), so mark it active in both
    const int p = par < 0 ? 0 : par;
    sd->st[p] = S;
    sd->st[p ^ 1] = S;
    *sd->result = S;
    active[p * n_active + slot] = 1;
    if (par < 0) active[(p ^ 1) * n_active + slot] = 1;
    if (ctl) {
      ctl->counter = 0;
      ctl->err = 0;
      ctl->round0 = p;
      ctl->round_end = p;
      ctl->nonfinite = 0;
    }
  }
  for (int q = threadIdx.x; q < b.nfaults; q += blockDim.x) const_cast<Fault*>(sd->faults)[q] = b.faults[q];
  for (int q = threadIdx.x; q < b.nlosses; q += blockDim.x) const_cast<LossEv*>(sd->losses)[q] = b.losses[q];
}

// ------------------------------------------------------------ host helpers
struct DeviceInfo {
  int sms = 0;
  int smem_optin = 0;
};
DeviceInfo device_info(int dev) {
  static std::mutex mu;
  static std::vector<DeviceInfo> cache;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)cache.size() <= dev) cache.resize(dev + 1);
  if (cache[dev].sms == 0) {
    cudaDeviceGetAttribute(&cache[dev].sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&cache[dev].smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  }
  return cache[dev];
}

// Per-row geometry of the latitude-longitude grid on the unit sphere (same
// definition, written out, as the problem statement in include/ftgcr.h).
void row_geometry(int nlon, int nlat, std::vector<double>& cx, std::vector<double>& cy, std::vector<double>& area) {
  const double dlam = 2.0 * kPi / nlon;
  const double dth = kPi / nlat;
  cx.resize(nlat);
  cy.resize(nlat);
  area.resize(nlat);
  for (int j = 0; j < nlat; ++j) {
    const double th = -0.5 * kPi + (j + 0.5) * dth;
    const double s_south = (j == 0) ? -1.0 : sin(-0.5 * kPi + j * dth);
    const double s_north = (j == nlat - 1) ? 1.0 : sin(-0.5 * kPi + (j + 1) * dth);
    cx[j] = dth / (cos(th) * dlam);
    cy[j] = (j == nlat - 1) ? 0.0 : cos(-0.5 * kPi + (j + 1) * dth) * dlam / dth;
    area[j] = dlam * (s_north - s_south);
  }
}


size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Dynamic shared memory of the persistent kernel for a solve with nt tiles.
// One-pass rounds: the tile's rows plus two halo rows (inner precision)
// followed by the line-solve constants of those rows.  Split rounds: the
// first pass holds the own rows and their constants, the second the rows with
// halos; the constants go after room for the halo rows when that fits (they
// then survive the second pass), else right after the own rows.  The mixed
// path's refinement phase holds the rows with halos in FP64.
struct SmemPlan {
  size_t bytes;
  long long cs_off;  // elements of the inner type
  int cs_clobber;
  int gconsts;  // FP64 line solve: factors read from global memory, not staged
  int sub_h;    // streamed solves: rows per sub-band of the split INIT / OUT rounds
  int nslot;    // streamed solves: stage buffers of the step rounds (stages in flight + 1)
};

// Streamed step rounds (mixed path, line preconditioner): the shared memory
// of a band of nlon columns.  Fixed part: three e rows and one row of line-
// solve constants; then stage buffers of kNVS rows of kCW floats (and their
// Tx leads): three (two stages in flight) where rows span at least two
// chunks and memory allows, else two.  The split INIT and OUT rounds of the
// same solve walk the band in sub-bands of sub_h rows that fit the same
// memory.  Returns false where two stage buffers do not fit.
bool stream_plan(int nlon, int k, size_t limit, SmemPlan* p) {
  (void)k;  // stages of more than kNVS operand rows are taken in sub-stages
  const int C = chunk_len(nlon);
  // piece-major rows: C a power of two from 32 to 256 (the line solve's
  // pieces are C / 8 elements in registers)
  if (nlon % 4 != 0 || C < 32 || C > 256 || (C & (C - 1))) return false;
  const size_t st = (size_t)row_stride(nlon), per_row = 32 * (size_t)C;
  const size_t prow = 32 * (size_t)(C + 4);  // a piece-major row
  const size_t fixed = 6 * prow * sizeof(float);
  const size_t buf = (size_t)kNVS * kCW * sizeof(float) + 8 * 16;
  int nbuf = (nlon > kCW && fixed + 3 * buf <= limit) ? 3 : 2;
  if (fixed + nbuf * buf > limit) return false;
  auto split_bytes = [&](size_t h) {
    return std::max({h * st * sizeof(float) + 3 * h * per_row * sizeof(float), (h + 2) * st * sizeof(float),
                     (h + 2) * st * sizeof(double)});
  };
  int sub = 0;
  for (int h = 1; h <= kMaxStreamRows; ++h)
    if (split_bytes((size_t)h) <= limit) sub = h;
  if (sub < 1) return false;
  p->bytes = std::max(fixed + (size_t)nbuf * buf, split_bytes((size_t)sub));
  p->cs_off = (long long)((size_t)sub * st);
  p->cs_clobber = 1;
  p->gconsts = 0;
  p->sub_h = sub;
  p->nslot = nbuf;
  return true;
}

SmemPlan smem_plan(int nlon, int nlat, int nt, int mixed, size_t elem, int precond, int split, size_t limit,
                   int gconsts = 0) {
  const size_t h = (size_t)((nlat + nt - 1) / nt);
  const size_t st = (size_t)row_stride(nlon);
  // chunk layout (FP32; FP64 rows of at least kChunkMinLon) or natural (FP64 serial solve)
  const size_t per_row = (mixed || nlon >= kChunkMinLon) ? 32 * (size_t)chunk_len(nlon) : (size_t)nlon;
  const size_t out = mixed ? (h + 2) * st * sizeof(double) : 0;
  const bool line = precond == FTGCR_PRECOND_LINE;
  SmemPlan p;
  p.gconsts = 0;
  p.sub_h = 0;
  p.nslot = 0;
  if (!split) {
    p.gconsts = line && !mixed && gconsts;
    // staged: three factor arrays per row; global: each row's factor ring
    const size_t consts = !line ? 0 : p.gconsts ? (h + 2) * (size_t)kRingStride * elem : 3 * (h + 2) * per_row * elem;
    p.bytes = std::max((h + 2) * st * elem + consts, out);
    p.cs_off = (long long)((h + 2) * st);
    p.cs_clobber = 0;
    return p;
  }
  const size_t consts = line ? 3 * h * per_row * elem : 0;
  const size_t roomy = std::max((h + 2) * st * elem + consts, out);
  if (roomy <= limit) {
    p.bytes = roomy;
    p.cs_off = (long long)((h + 2) * st);
    p.cs_clobber = 0;
  } else {
    p.bytes = std::max({h * st * elem + consts, (h + 2) * st * elem, out});
    p.cs_off = (long long)(h * st);
    p.cs_clobber = 1;
  }
  return p;
}

// Row bands and round structure of a solve.  Equal-height row bands: the
// round takes as long as the tallest band, so use the fewest bands of that
// height (e.g. 512 rows on 152 SMs: 128 x 4), as tall as shared memory allows.
// Split rounds (mixed path, line preconditioner) when shared memory, not the
// SM count, cuts one-pass tiles below three rows (each tile would then
// recompute at least twice its own rows as halo), or when one row with its
// halo rows and their constants does not fit at all.
// Mixed solves of at least this many points stream their step rounds by
// default: their Krylov vectors (about 16 FP32 vectors of N) far outgrow the
// 129 MB L2, so a round is bound by HBM rather than by L2 latency.  Smaller
// solves run faster in one-pass rounds (measured per inner step: 2048 x 1024
// 83 us in one-pass rounds against 94 streamed; 4096 x 2048 247 streamed
// against 401 in split rounds).
constexpr long long kStreamMinPoints = 4LL * 1024 * 1024;

// Streamed step rounds: one band per SM (at most kMaxStreamRows rows).
int stream_tiles(int nlat, int tiles, int sms) {
  int nt = tiles > 0 ? std::min(tiles, nlat) : std::min(nlat, sms);
  if ((nlat + nt - 1) / nt > kMaxStreamRows) nt = (nlat + kMaxStreamRows - 1) / kMaxStreamRows;
  return nt;
}

void choose_tiling(int nlon, int nlat, int mixed, size_t elem, int precond, int flags, int tiles, int sms,
                   size_t limit, int k, int* nt_out, int* split_out, int* gconsts_out) {
  const int hpar = (nlat + sms - 1) / sms;  // band height the SM count alone gives
  auto fit = [&](int split, int gc = 0) {
    int nt = (nlat + hpar - 1) / hpar;
    while (nt < nlat && smem_plan(nlon, nlat, nt, mixed, elem, precond, split, limit, gc).bytes > limit)
      nt = std::min(nlat, nt + sms);
    return nt;
  };
  // FP64 line solve: its factors are read from global memory when staging
  // them would cut the bands below what the SM count gives (wide rows).  The
  // row solves are chains of dependent FP64 operations that cost the same
  // for all the rows of a tile side by side in lanes, so a CTA that walks
  // several thin tiles a round pays the chains once per tile.
  *gconsts_out = 0;
  if (!mixed && precond == FTGCR_PRECOND_LINE) {
    if (tiles > 0) {
      *gconsts_out = smem_plan(nlon, nlat, std::min(tiles, nlat), mixed, elem, precond, 0, limit).bytes > limit;
    } else {
      const int nt0 = fit(0);
      *gconsts_out = smem_plan(nlon, nlat, nt0, mixed, elem, precond, 0, limit).bytes > limit ||
                     (nlat + nt0 - 1) / nt0 < hpar;
    }
    *split_out = 0;
    *nt_out = tiles > 0 ? std::min(tiles, nlat) : fit(0, *gconsts_out);
    return;
  }
  int split = 0;
  if (mixed && precond == FTGCR_PRECOND_LINE) {
    SmemPlan sp;
    const bool can_stream = stream_plan(nlon, k, limit, &sp);
    if ((flags & FTGCR_FLAG_STREAMED_ROUNDS) ||
        (!(flags & (FTGCR_FLAG_SPLIT_ROUNDS | FTGCR_FLAG_FUSED_ROUNDS)) && can_stream &&
         (long long)nlon * nlat >= kStreamMinPoints)) {
      *split_out = can_stream ? 2 : -1;  // -1: streamed rounds asked for but impossible
      *nt_out = stream_tiles(nlat, tiles, sms);
      return;
    }
    if (flags & FTGCR_FLAG_SPLIT_ROUNDS)
      split = 1;
    else if (!(flags & FTGCR_FLAG_FUSED_ROUNDS)) {
      const int nt1 = tiles > 0 ? std::min(tiles, nlat) : fit(0);
      const int h1 = (nlat + nt1 - 1) / nt1;
      const bool fits = smem_plan(nlon, nlat, nt1, mixed, elem, precond, 0, limit).bytes <= limit;
      split = !fits || (h1 < hpar && h1 < 3);
    }
  }
  *split_out = split;
  *nt_out = tiles > 0 ? std::min(tiles, nlat) : fit(split);
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FTGCR_OK;
  if (e == cudaErrorMemoryAllocation) return FTGCR_ERR_OOM;
  return FTGCR_ERR_CUDA;
}

#define CK(x)                                  \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)

constexpr int kStaticSmemReserve = 20 * 1024;  // KernelSmem and friends

}  // namespace

// ------------------------------------------------------------ the handle
struct ftgcr_handle {
  int dev = 0;
  int nlon = 0, nlat = 0, k = 0, precision = 0, precond = 0, nt = 0, C = 0;
  long long N = 0, max_steps = 0;
  double tol = 0, mu = 0, inner_tol = 0;
  int max_outer = 0;
  int flags = 0;
  unsigned char* pool = nullptr;
  size_t pool_bytes = 0;
  size_t backup_bytes = 0;
  // FP64 operator (always)
  double *Tx64 = nullptr, *Ty64 = nullptr, *muA64 = nullptr;
  double *stageR = nullptr, *stageX = nullptr;  // host-pointer staging
  void* sdev = nullptr;                        // SolveDev<T>* on the device
  void** sdev_arr = nullptr;                   // device array holding sdev
  int* nt_dev = nullptr;
  int* active = nullptr;                       // [2]
  int* diag = nullptr;                         // [grid][4] per-CTA progress (timeout report)
  LaunchCtl* ctl = nullptr;
  SolveState* result = nullptr;
  SolveState* h_result = nullptr;              // pinned
  LaunchCtl* h_ctl = nullptr;                  // pinned
  SolveDev<double> sd64{};
  SolveDev<float> sd32{};
  size_t smem = 0;
  int split = 0;  // split rounds (see choose_tiling)
  int wide = 0;   // runs in the wide-row kernel instance (split rounds, or FP64 factors from global memory)
  int noalloc = 0;  // the record of a no-allocation solve (its pool is the static scratch array)
  SmemPlan plan{};
  int grid = 0;
  cudaStream_t last_stream = nullptr;
  int solved = 0;
  int last_status = FTGCR_ERR_STATE;
};

namespace {

// Compile-time bound on the Krylov directions of the kernel instance.
int kbound(int k) { return k <= 4 ? 4 : (k <= 8 ? 8 : 16); }

// The persistent kernel instances live in their own translation units
// (ftgcr_k4.cu, ftgcr_k8.cu, ftgcr_k16.cu, their mixed split-round twins
// ftgcr_k*s.cu and their FP64 wide-row twins ftgcr_k*w.cu) so that they
// compile in parallel.  wide: the wide-row instance.
template <typename T>
const void* kernel_ptr(int kb, int wide) {
  return ftgcr::persistent_kernel_ptr(kb, sizeof(T) == 8, wide);
}

// The dynamic shared memory attribute of a kernel is process-wide: only ever
// raise it, so that a handle created later never shrinks what an earlier one
// needs.
template <typename T>
int configure_kernel(int kb, int split, size_t smem) {
  static std::mutex mu;
  static std::vector<std::pair<const void*, size_t>> set;
  std::lock_guard<std::mutex> lk(mu);
  const void* f = kernel_ptr<T>(kb, split);
  for (auto& e : set)
    if (e.first == f) {
      if (e.second >= smem) return FTGCR_OK;
      CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      e.second = smem;
      return FTGCR_OK;
    }
  CK(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  set.emplace_back(f, smem);
  return FTGCR_OK;
}

// Resident CTAs per SM of a kernel instance at a dynamic shared memory size,
// cached (the same answer every time; a batch launch being captured into a
// CUDA graph then makes no query).
template <typename T>
int occupancy(int kb, int split, size_t smem, int* occ) {
  static std::mutex mu;
  static std::map<std::pair<const void*, size_t>, int> known;
  const void* f = kernel_ptr<T>(kb, split);
  std::lock_guard<std::mutex> lk(mu);
  auto it = known.find({f, smem});
  if (it != known.end()) {
    *occ = it->second;
    return FTGCR_OK;
  }
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, f, kThreads, smem));
  known[{f, smem}] = *occ;
  return FTGCR_OK;
}

bool is_device_ptr(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int validate_plan(const ftgcr_handle* h, const ftgcr_fault_plan* plan) {
  if (!plan) return FTGCR_OK;
  if (plan->nlosses < 0 || plan->nlosses > FTGCR_MAX_LOSSES || (plan->nlosses > 0 && !plan->losses))
    return FTGCR_ERR_ARG;
  for (int q = 0; q < plan->nlosses; ++q) {
    const ftgcr_loss& l = plan->losses[q];
    if (l.step < 1 || l.nranks < 1 || l.rank < 0 || l.rank >= l.nranks || l.count < 0) return FTGCR_ERR_ARG;
  }
  if (plan->n == 0) return FTGCR_OK;
  if (plan->n < 0 || plan->n > FTGCR_MAX_FAULTS || !plan->faults) return FTGCR_ERR_ARG;
  const int maxbit = h->precision == FTGCR_MIXED ? 31 : 63;
  for (int q = 0; q < plan->n; ++q) {
    const ftgcr_fault& f = plan->faults[q];
    if (f.vec < 0 || f.vec > FTGCR_VEC_E || f.index < 0 || f.index >= h->N || f.bit < 0 || f.bit > maxbit ||
        f.step < 1)
      return FTGCR_ERR_ARG;
  }
  return FTGCR_OK;
}

// Carve every allocation of a handle out of one pool (or just count bytes).
template <typename T>
size_t layout(ftgcr_handle* h, unsigned char* base, SolveDev<T>* sd) {
  size_t off = 0;
  const long long N = h->N;
  const int nlat = h->nlat, k = h->k, C = h->C;
  auto take = [&](size_t bytes) -> unsigned char* {
    unsigned char* p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  const size_t vT = sizeof(T) * N, v64 = sizeof(double) * N;
  const bool fp64 = std::is_same<T, double>::value;
  // preconditioner arrays: FP64 natural [N] (+ u), FP32 chunk layout [nlat][32 C]
  const size_t lcn = (h->precond == FTGCR_PRECOND_LINE) ? (fp64 ? (size_t)N : (size_t)nlat * 32 * C)
                                                        : (h->precond == FTGCR_PRECOND_JACOBI ? (size_t)N : 1);
  h->Tx64 = (double*)take(v64);
  h->Ty64 = (double*)take(v64);
  h->muA64 = (double*)take(sizeof(double) * nlat);
  sd->Tx = (const T*)(std::is_same<T, double>::value ? (void*)h->Tx64 : (void*)take(vT));
  sd->Ty = (const T*)(std::is_same<T, double>::value ? (void*)h->Ty64 : (void*)take(vT));
  sd->muA = (const T*)(std::is_same<T, double>::value ? (void*)h->muA64 : (void*)take(sizeof(T) * nlat));
  sd->lc = (const T*)take(sizeof(T) * lcn);
  sd->lw = (const T*)take(sizeof(T) * lcn);
  sd->lz = (const T*)take(sizeof(T) * lcn);
  sd->lu = (const T*)(fp64 && h->precond == FTGCR_PRECOND_LINE ? take(sizeof(T) * lcn) : nullptr);
  sd->lrow = (const T*)take(sizeof(T) * 4 * nlat);
  // FP64 chunked row solves: the factors again in the chunk layout
  // (not with FTGCR_FLAG_ORACLE_ORDER: the oracle's serial order on every row;
  // the shared-memory plan was sized for the larger chunk layout)
  const bool chunk = fp64 && h->precond == FTGCR_PRECOND_LINE && h->nlon >= kChunkMinLon && !h->noalloc &&
                     !(h->flags & FTGCR_FLAG_ORACLE_ORDER);
  sd->lchunk = chunk ? 1 : 0;
  sd->lcc = chunk ? (const T*)take(sizeof(T) * 32 * (size_t)C * nlat) : sd->lc;
  sd->lwc = chunk ? (const T*)take(sizeof(T) * 32 * (size_t)C * nlat) : sd->lw;
  sd->lzc = chunk ? (const T*)take(sizeof(T) * 32 * (size_t)C * nlat) : sd->lz;
  // streamed solves: the FP32 constants again in the piece-major layout
  const bool piece = !fp64 && h->split == 2;
  sd->lcp = piece ? (const T*)take(sizeof(T) * 32 * (size_t)(C + 4) * nlat) : nullptr;
  sd->lwp = piece ? (const T*)take(sizeof(T) * 32 * (size_t)(C + 4) * nlat) : nullptr;
  sd->lzp = piece ? (const T*)take(sizeof(T) * 32 * (size_t)(C + 4) * nlat) : nullptr;
  size_t before = off;
  for (int q = 0; q < 3; ++q) sd->phi[q] = (T*)take(vT);
  for (int q = 0; q < 3; ++q) sd->r[q] = (T*)take(vT);
  sd->e[0] = (T*)take(vT);
  sd->Le[0] = (T*)take(vT);
  if (std::is_same<T, float>::value) {  // mixed path: fused steps double-buffer e, L(e)
    sd->e[1] = (T*)take(vT);
    sd->Le[1] = (T*)take(vT);
  } else {
    sd->e[1] = sd->e[0];
    sd->Le[1] = sd->Le[0];
  }
  for (int s = 0; s < kNSlot; ++s) {
    sd->p[s] = s < k + 2 ? (T*)take(vT) : nullptr;
    sd->Lp[s] = s < k + 2 ? (T*)take(vT) : nullptr;
  }
  (void)before;
  h->backup_bytes = 4 * vT;
  sd->Rin = (T*)(std::is_same<T, float>::value ? take(vT) : nullptr);
  sd->xbuf[0] = (double*)(std::is_same<T, float>::value ? take(v64) : nullptr);
  sd->xbuf[1] = (double*)(std::is_same<T, float>::value ? take(v64) : nullptr);
  h->stageR = (double*)take(v64);
  h->stageX = (double*)take(v64);
  sd->part = (double*)take(sizeof(double) * 2 * h->nt * kPartStride);  // [2 parities][nt][kNPart pairs]
  sd->st = (SolveState*)take(sizeof(SolveState) * 2);
  sd->result = (SolveState*)take(sizeof(SolveState));
  sd->faults = (const Fault*)take(sizeof(Fault) * kMaxFaults);
  sd->losses = (const LossEv*)take(sizeof(LossEv) * kMaxLosses);
  sd->patchval = (double*)take(sizeof(double) * kMaxFaults);
  h->sdev = take(sizeof(SolveDev<T>));
  h->sdev_arr = (void**)take(sizeof(void*));
  h->nt_dev = (int*)take(sizeof(int));
  h->active = (int*)take(sizeof(int) * 2);
  h->diag = (int*)take(sizeof(int) * 4 * 4096);
  h->ctl = (LaunchCtl*)take(sizeof(LaunchCtl));
  h->result = sd->result;
  return off;
}

// Face coefficients and line-preconditioner factorisation of a handle from the
// cell-centred coefficient D (device pointer), enqueued on `st`: per-row
// geometry on the host (libm), everything per element on the device.  Used
// at create and whenever a handle is reused for new coefficients (serving).
// Scratch is stream-ordered (cudaMallocAsync / cudaFreeAsync).
template <typename T>
int setup_coefficients(ftgcr_handle* h, const SolveDev<T>& sd, const double* Dd, cudaStream_t st) {
  std::vector<double> geo;
  {
    std::vector<double> cx, cy, area;
    row_geometry(h->nlon, h->nlat, cx, cy, area);
    geo.insert(geo.end(), cx.begin(), cx.end());
    geo.insert(geo.end(), cy.begin(), cy.end());
    geo.insert(geo.end(), area.begin(), area.end());
  }
  const bool mixed = std::is_same<T, float>::value;
  const size_t geo_bytes = align256(sizeof(double) * 3 * h->nlat);
  const size_t tmp_bytes = mixed ? sizeof(double) * (4 * (size_t)h->N + 4 * h->nlat) : 0;
  unsigned char* scratch = nullptr;
  CK(cudaMallocAsync((void**)&scratch, geo_bytes + tmp_bytes, st));
  double* dcx = (double*)scratch;
  CK(cudaMemcpyAsync(dcx, geo.data(), sizeof(double) * 3 * h->nlat, cudaMemcpyHostToDevice, st));
  k_face_coeffs<<<1024, 256, 0, st>>>(h->nlon, h->nlat, Dd, dcx, dcx + h->nlat, dcx + 2 * h->nlat, h->mu, h->Tx64,
                                      h->Ty64, h->muA64, mixed ? (float*)sd.Tx : nullptr,
                                      mixed ? (float*)sd.Ty : nullptr, mixed ? (float*)sd.muA : nullptr);
  CK(cudaGetLastError());
  // FP64 factors: into the handle (FP64 path) or scratch (mixed path)
  double *l64, *w64, *u64, *z64, *r64;
  if (!mixed) {
    l64 = (double*)sd.lc;
    w64 = (double*)sd.lw;
    u64 = (double*)sd.lu;
    z64 = (double*)sd.lz;
    r64 = (double*)sd.lrow;
  } else {
    double* tmp = (double*)(scratch + geo_bytes);
    l64 = tmp;
    w64 = tmp + h->N;
    u64 = tmp + 2 * h->N;
    z64 = tmp + 3 * h->N;
    r64 = tmp + 4 * h->N;
  }
  const bool chunk = !mixed && sd.lchunk;
  const int frc = launch_line_factor(h->nlon, h->nlat, h->C, h->precond, h->Tx64, h->Ty64, h->muA64, l64, w64, u64,
                                     z64, r64, mixed ? (float*)sd.lc : nullptr, mixed ? (float*)sd.lw : nullptr,
                                     mixed ? (float*)sd.lz : nullptr, mixed ? (float*)sd.lrow : nullptr, st,
                                     chunk ? (double*)sd.lcc : nullptr, chunk ? (double*)sd.lwc : nullptr,
                                     chunk ? (double*)sd.lzc : nullptr, mixed ? (float*)sd.lcp : nullptr,
                                     mixed ? (float*)sd.lwp : nullptr, mixed ? (float*)sd.lzp : nullptr);
  if (frc) return frc;
  CK(cudaFreeAsync(scratch, st));
  return FTGCR_OK;
}

template <typename T>
int create_impl(ftgcr_handle* h, const double* D_host_or_dev, bool D_on_device) {
  SolveDev<T> sd{};
  const size_t bytes = layout<T>(h, nullptr, &sd);
  if (cudaMalloc(&h->pool, bytes) != cudaSuccess) {
    cudaGetLastError();
    return FTGCR_ERR_OOM;
  }
  h->pool_bytes = bytes;
  CK(cudaMemset(h->pool, 0, bytes));
  layout<T>(h, h->pool, &sd);
  sd.nlon = h->nlon;
  sd.nlat = h->nlat;
  sd.k = h->k;
  sd.nt = h->nt;
  sd.nt_hmax = (h->nlat + h->nt - 1) / h->nt;
  sd.C = h->C;
  sd.precond = h->precond;
  sd.mixed = std::is_same<T, float>::value ? 1 : 0;
  sd.nfaults = 0;
  sd.N = h->N;
  sd.max_steps = h->max_steps;
  sd.max_outer = h->max_outer;
  sd.tol2 = h->tol * h->tol;
  sd.inner_tol2 = h->inner_tol * h->inner_tol;
  sd.protect = (h->flags & FTGCR_FLAG_UNPROTECTED) ? 0 : 1;
  sd.zero_guess = (h->flags & FTGCR_FLAG_ZERO_GUESS) ? 1 : 0;
  sd.oracle_order = (h->flags & FTGCR_FLAG_ORACLE_ORDER) ? 1 : 0;
  sd.split = h->split;
  sd.cs_off = (int)h->plan.cs_off;
  sd.cs_clobber = h->plan.cs_clobber;
  sd.cs_global = h->plan.gconsts;
  sd.sub_h = h->plan.sub_h;
  sd.nslot = h->plan.nslot;
  sd.Tx64 = h->Tx64;
  sd.Ty64 = h->Ty64;
  sd.muA64 = h->muA64;

  // face coefficients and factorisation (device)
  double* dD = nullptr;
  const double* Dd = D_host_or_dev;
  if (!D_on_device) {
    CK(cudaMalloc(&dD, sizeof(double) * h->N));
    CK(cudaMemcpy(dD, D_host_or_dev, sizeof(double) * h->N, cudaMemcpyHostToDevice));
    Dd = dD;
  }
  int src = setup_coefficients<T>(h, sd, Dd, nullptr);
  if (src) return src;
  CK(cudaDeviceSynchronize());
  if (dD) cudaFree(dD);
  const bool mixed = std::is_same<T, float>::value;

  CK(cudaMemcpy(h->sdev, &sd, sizeof sd, cudaMemcpyHostToDevice));
  void* sp = h->sdev;
  CK(cudaMemcpy(h->sdev_arr, &sp, sizeof(void*), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(h->nt_dev, &h->nt, sizeof(int), cudaMemcpyHostToDevice));
  if constexpr (std::is_same<T, float>::value)
    h->sd32 = sd;
  else
    h->sd64 = sd;

  (void)mixed;
  h->smem = h->plan.bytes;
  int rc = configure_kernel<T>(kbound(h->k), h->wide, std::max<size_t>(h->smem, 1));
  if (rc) return rc;
  int occ = 0;
  rc = occupancy<T>(kbound(h->k), h->wide, h->smem, &occ);
  if (rc) return rc;
  if (occ < 1) return FTGCR_ERR_ARG;
  {
    // the per-thread stack must hold the kernel's spill frame
    cudaFuncAttributes fa;
    CK(cudaFuncGetAttributes(&fa, kernel_ptr<T>(kbound(h->k), h->wide)));
    size_t cur = 0;
    CK(cudaDeviceGetLimit(&cur, cudaLimitStackSize));
    if (fa.localSizeBytes + 256 > cur) CK(cudaDeviceSetLimit(cudaLimitStackSize, fa.localSizeBytes + 256));
  }
  const DeviceInfo di = device_info(h->dev);
  h->grid = std::min(h->nt, di.sms * occ);
  CK(cudaMallocHost(&h->h_result, sizeof(SolveState)));
  CK(cudaMallocHost(&h->h_ctl, sizeof(LaunchCtl)));
  return FTGCR_OK;
}

// Developer trace (FTGCR_TRACE=<csv path>): per-round timestamps of every
// CTA of the next launches, written after each blocking solve.
struct TraceBuf {
  TraceEnt* d = nullptr;
  int rounds = 0, grid = 0;
  const char* path = nullptr;
};
TraceBuf& trace_buf() {
  static TraceBuf t;
  return t;
}
TraceEnt* trace_ptr(int grid, int* rounds) {
  TraceBuf& t = trace_buf();
  t.path = getenv("FTGCR_TRACE");
  if (!t.path || !*t.path) return nullptr;
  const int want = 4096;
  if (!t.d || t.grid < grid) {
    if (t.d) cudaFree(t.d);
    if (cudaMalloc(&t.d, sizeof(TraceEnt) * (size_t)want * grid) != cudaSuccess) {
      cudaGetLastError();
      t.d = nullptr;
      return nullptr;
    }
    t.rounds = want;
    t.grid = grid;
  }
  cudaMemset(t.d, 0, sizeof(TraceEnt) * (size_t)t.rounds * t.grid);
  *rounds = t.rounds;
  return t.d;
}
void trace_dump(int grid) {
  TraceBuf& t = trace_buf();
  if (!t.d || !t.path || !*t.path) return;
  std::vector<TraceEnt> h((size_t)t.rounds * t.grid);
  cudaMemcpy(h.data(), t.d, h.size() * sizeof(TraceEnt), cudaMemcpyDeviceToHost);
  FILE* f = fopen(t.path, "w");
  if (!f) return;
  fprintf(f, "round,cta,kind,items,t0,t1,t2,t3,s0,s1,s2\n");
  for (int r = 0; r < t.rounds; ++r)
    for (int b = 0; b < grid; ++b) {
      const TraceEnt& e = h[(size_t)r * t.grid + b];
      if (e.t3 == 0) continue;
      fprintf(f, "%d,%d,%d,%d,%llu,%llu,%llu,%llu,%llu,%llu,%llu\n", r, b, e.kind, e.items, e.t0, e.t1, e.t2, e.t3,
              e.s0, e.s1, e.s2);
    }
  fclose(f);
}

template <typename T>
int launch_persistent(int kb, SolveDev<T>* const* solves, const int* nt, int* active, int n, LaunchCtl* ctl,
                      int* diag, int max_rounds, int grid, size_t smem, int split, cudaStream_t st) {
  BatchArgs<T> a;
  a.solves = solves;
  a.nt = nt;
  a.active = active;
  a.n = n;
  a.ctl = ctl;
  a.max_rounds = max_rounds;
  a.trace = trace_ptr(grid, &a.trace_rounds);
  a.diag = diag;
  void* args[] = {&a};
  CK(cudaLaunchCooperativeKernel(kernel_ptr<T>(kb, split), dim3(grid), dim3(kThreads), args, smem, st));
  return FTGCR_OK;
}

BeginArgs begin_args(const ftgcr_handle* h, const double* R, const double* x0, double* xout,
                     const ftgcr_fault_plan* plan) {
  BeginArgs b;
  memset(&b, 0, sizeof b);
  b.R = R;
  b.x0 = x0;
  b.xout = xout;
  b.nfaults = plan ? plan->n : 0;
  b.nlosses = plan && plan->losses ? plan->nlosses : 0;
  b.max_steps = h->max_steps;
  for (int q = 0; q < b.nfaults; ++q) memcpy(&b.faults[q], &plan->faults[q], sizeof(Fault));
  for (int q = 0; q < b.nlosses; ++q) memcpy(&b.losses[q], &plan->losses[q], sizeof(LossEv));
  return b;
}

template <typename T>
int solve_async_impl(ftgcr_handle* h, const double* R, const double* x0, double* xout, const ftgcr_fault_plan* plan,
                     cudaStream_t st, bool check_finite = false) {
  const BeginArgs b = begin_args(h, R, x0, xout, plan);
  k_begin_solve<T><<<1, 64, 0, st>>>((SolveDev<T>*)h->sdev, b, h->active, 1, 0, 0, h->ctl,
                                     check_finite ? h->ctl : nullptr);
  CK(cudaGetLastError());
  // every inner step takes two rounds, every refinement sweep a few more
  const int max_rounds = (int)std::min<long long>(1 << 30, 2 * h->max_steps + 8 * ((long long)h->max_outer + 2) + 16);
  int rc = launch_persistent<T>(kbound(h->k), (SolveDev<T>* const*)h->sdev_arr, h->nt_dev, h->active, 1, h->ctl,
                                h->diag, max_rounds, h->grid, h->smem, h->wide, st);
  if (rc) return rc;
  CK(cudaMemcpyAsync(h->h_result, h->result, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(h->h_ctl, h->ctl, sizeof(LaunchCtl), cudaMemcpyDeviceToHost, st));
  h->last_stream = st;
  h->solved = 1;
  return FTGCR_OK;
}

// Several independent solves in one persistent launch.  Each solve keeps its
// own handle's tiling and reduction order, so its arithmetic is bitwise that
// of a lone solve; the launch only interleaves the solves' tiles over the
// CTAs.  The launch's own arrays (solve pointers, tile counts, active flags,
// control block, progress record) are stream-ordered allocations freed after
// the launch, and the solve table is written by a kernel from its parameters
// (no copy from host memory), so a batch captures into a CUDA graph.
template <typename T>
int solve_batch_impl(ftgcr_handle* const* hs, const double* const* rhs, double* const* x,
                     const ftgcr_fault_plan* const* plans, int n, cudaStream_t st) {
  int kb = 4;
  size_t smem = 1;
  long long max_steps = 0, total_tiles = 0;
  int max_outer = 0, split = 0;
  for (int i = 0; i < n; ++i) {
    split = std::max(split, hs[i]->wide);
    kb = std::max(kb, kbound(hs[i]->k));
    smem = std::max(smem, hs[i]->smem);
    max_steps = std::max(max_steps, hs[i]->max_steps);
    max_outer = std::max(max_outer, hs[i]->max_outer);
    total_tiles += hs[i]->nt;
  }
  int rc = configure_kernel<T>(kb, split, smem);
  if (rc) return rc;
  int occ = 0;
  rc = occupancy<T>(kb, split, smem, &occ);
  if (rc) return rc;
  if (occ < 1) return FTGCR_ERR_ARG;
  const DeviceInfo di = device_info(hs[0]->dev);
  const int grid = (int)std::min<long long>(total_tiles, (long long)di.sms * occ);
  const size_t b_solves = align256(sizeof(void*) * n), b_nt = align256(sizeof(int) * n),
               b_act = align256(sizeof(int) * 2 * n), b_ctl = align256(sizeof(LaunchCtl)),
               b_diag = align256(sizeof(int) * 4 * grid);
  unsigned char* buf = nullptr;
  CK(cudaMallocAsync((void**)&buf, b_solves + b_nt + b_act + b_ctl + b_diag, st));
  void** d_solves = (void**)buf;
  int* d_nt = (int*)(buf + b_solves);
  int* d_act = (int*)(buf + b_solves + b_nt);
  LaunchCtl* d_ctl = (LaunchCtl*)(buf + b_solves + b_nt + b_act);
  int* d_diag = (int*)(buf + b_solves + b_nt + b_act + b_ctl);
  for (int off = 0; off < n; off += kTableChunk) {
    BatchTable tb;
    tb.n = std::min(kTableChunk, n - off);
    tb.off = off;
    for (int i = 0; i < tb.n; ++i) {
      tb.sdev[i] = hs[off + i]->sdev;
      tb.nt[i] = hs[off + i]->nt;
    }
    k_fill_table<<<1, kTableChunk, 0, st>>>(tb, d_solves, d_nt);
    CK(cudaGetLastError());
  }
  CK(cudaMemsetAsync(d_act, 0, sizeof(int) * 2 * n, st));
  for (int i = 0; i < n; ++i) {
    const BeginArgs b = begin_args(hs[i], rhs[i], x[i], x[i], plans ? plans[i] : nullptr);
    k_begin_solve<T><<<1, 64, 0, st>>>((SolveDev<T>*)hs[i]->sdev, b, d_act, n, i, 0, i == 0 ? d_ctl : nullptr);
    CK(cudaGetLastError());
  }
  const int max_rounds = (int)std::min<long long>(1 << 30, 2 * max_steps + 8 * ((long long)max_outer + 2) + 16);
  rc = launch_persistent<T>(kb, (SolveDev<T>* const*)d_solves, d_nt, d_act, n, d_ctl, d_diag, max_rounds, grid, smem,
                            split, st);
  if (rc) {
    cudaFreeAsync(buf, st);
    return rc;
  }
  for (int i = 0; i < n; ++i) {
    CK(cudaMemcpyAsync(hs[i]->h_result, hs[i]->result, sizeof(SolveState), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(hs[i]->h_ctl, d_ctl, sizeof(LaunchCtl), cudaMemcpyDeviceToHost, st));
    hs[i]->last_stream = st;
    hs[i]->solved = 1;
  }
  CK(cudaFreeAsync(buf, st));
  return FTGCR_OK;
}

// ------------------------------------------------------------ slot tables
// The launch arrays of a resumable persistent launch, kept across launches:
// per slot the solve descriptor and tile count, the double-buffered active
// flags, and the control block whose round counter carries the round parity
// from one launch to the next.
struct SlotTableImpl {
  int precision = 0, n = 0, dev = 0;
  long long round = 0;  // index of the next round to run
  unsigned char* buf = nullptr;
  void** d_solves = nullptr;
  int* d_nt = nullptr;
  int* d_act = nullptr;
  LaunchCtl* d_ctl = nullptr;
  int* d_diag = nullptr;
  LaunchCtl* h_ctl_in = nullptr;   // pinned: control block written before a launch
  LaunchCtl* h_ctl_out = nullptr;  // pinned: control block read back after it
  int* h_act = nullptr;            // pinned: active flags read back after it
  SolveState* d_results = nullptr;  // [n] result records gathered after a launch
  SolveState* h_results = nullptr;  // pinned: their copy
  int grid_cap = 0;
  std::vector<ftgcr_handle*> slot;
  std::vector<char> launched;  // slots occupied when the last launch was enqueued
};

// The result records of the solves a table launch ran (mask bit s: slot s was
// occupied), gathered into one array so that the scheduler reads them back
// with a single copy.
struct SlotMask {
  unsigned int bits[32];  // 1024 slots
};
template <typename T>
__global__ void k_gather_results(SolveDev<T>* const* solves, SlotMask mask, int n, SolveState* out) {
  constexpr int W = sizeof(SolveState) / sizeof(int);
  static_assert(sizeof(SolveState) % sizeof(int) == 0, "whole words");
  for (int s = blockIdx.x; s < n; s += gridDim.x) {
    if (!((mask.bits[s >> 5] >> (s & 31)) & 1u)) continue;
    const int* src = reinterpret_cast<const int*>(solves[s]->result);
    int* dst = reinterpret_cast<int*>(out + s);
    for (int q = threadIdx.x; q < W; q += blockDim.x) dst[q] = __ldcg(src + q);
  }
}

template <typename T>
int table_run_impl(SlotTableImpl* t, int max_rounds, cudaStream_t st) {
  int kb = 4;
  size_t smem = 1;
  long long tiles = 0;
  int split = 0;
  for (ftgcr_handle* h : t->slot)
    if (h) {
      split = std::max(split, h->wide);
      kb = std::max(kb, kbound(h->k));
      smem = std::max(smem, h->smem);
      tiles += h->nt;
    }
  if (tiles == 0) return FTGCR_OK;
  int rc = configure_kernel<T>(kb, split, smem);
  if (rc) return rc;
  int occ = 0;
  rc = occupancy<T>(kb, split, smem, &occ);
  if (rc) return rc;
  if (occ < 1) return FTGCR_ERR_ARG;
  const int grid = (int)std::min<long long>({tiles, (long long)device_info(t->dev).sms * occ, (long long)t->grid_cap});
  for (int s = 0; s < t->n; ++s) t->launched[s] = t->slot[s] != nullptr;
  t->h_ctl_in->counter = 0;
  t->h_ctl_in->err = 0;
  t->h_ctl_in->round0 = t->round;
  t->h_ctl_in->round_end = t->round;
  t->h_ctl_in->nonfinite = 0;
  CK(cudaMemcpyAsync(t->d_ctl, t->h_ctl_in, sizeof(LaunchCtl), cudaMemcpyHostToDevice, st));
  rc = launch_persistent<T>(kb, (SolveDev<T>* const*)t->d_solves, t->d_nt, t->d_act, t->n, t->d_ctl, t->d_diag,
                            max_rounds, grid, smem, split, st);
  if (rc) return rc;
  CK(cudaMemcpyAsync(t->h_ctl_out, t->d_ctl, sizeof(LaunchCtl), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(t->h_act, t->d_act, sizeof(int) * 2 * t->n, cudaMemcpyDeviceToHost, st));
  SlotMask mask;
  memset(&mask, 0, sizeof mask);
  for (int s = 0; s < t->n; ++s)
    if (t->launched[s]) mask.bits[s >> 5] |= 1u << (s & 31);
  k_gather_results<T><<<std::min(t->n, 128), 128, 0, st>>>((SolveDev<T>* const*)t->d_solves, mask, t->n,
                                                            t->d_results);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(t->h_results, t->d_results, sizeof(SolveState) * t->n, cudaMemcpyDeviceToHost, st));
  return FTGCR_OK;
}

void report_timeout(const ftgcr_handle* h) {
  std::vector<int> d((size_t)h->grid * 4);
  if (cudaMemcpy(d.data(), h->diag, d.size() * sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return;
  fprintf(stderr, "ftgcr: grid barrier timeout (code %d); per-CTA round/kind/checkpoint/items:\n", h->h_ctl->err);
  for (int b = 0; b < h->grid; ++b)
    fprintf(stderr, "  cta %d: round %d kind %d checkpoint %d items %d\n", b, d[4 * b], d[4 * b + 1], d[4 * b + 2],
            d[4 * b + 3]);
}

int status_from_result(const ftgcr_handle* h) {
  if (h->h_result->refused) return FTGCR_ERR_ARG;
  if (h->h_ctl->err) {
    report_timeout(h);
    return FTGCR_ERR_TIMEOUT;
  }
  const SolveState& S = *h->h_result;
  if (S.active) return FTGCR_ERR_CUDA;
  return S.status == ST_CONVERGED ? FTGCR_OK : FTGCR_NOT_CONVERGED;
}

}  // namespace

// ------------------------------------------------------------ C ABI
extern "C" {

const char* ftgcr_error_string(int status) {
  switch (status) {
    case FTGCR_OK: return "ok";
    case FTGCR_NOT_CONVERGED: return "not converged (step limit reached)";
    case FTGCR_ERR_ARG: return "invalid argument";
    case FTGCR_ERR_OOM: return "device out of memory";
    case FTGCR_ERR_CUDA: return "CUDA error";
    case FTGCR_ERR_TIMEOUT: return "grid barrier timed out";
    case FTGCR_ERR_BUDGET: return "request exceeds the memory budget";
    case FTGCR_ERR_STATE: return "call out of order";
    default: return "unknown status";
  }
}

static int check_grid(const ftgcr_grid* g, int32_t k, double tol) {
  if (!g) return FTGCR_ERR_ARG;
  if (g->nlon < 3 || g->nlat < 1 || g->nlon > (1 << 20) || g->nlat > (1 << 20)) return FTGCR_ERR_ARG;
  if (!(g->mu >= 0.0) || !std::isfinite(g->mu)) return FTGCR_ERR_ARG;
  if (g->precision != FTGCR_FP64 && g->precision != FTGCR_MIXED) return FTGCR_ERR_ARG;
  if (g->precond < FTGCR_PRECOND_LINE || g->precond > FTGCR_PRECOND_IDENTITY) return FTGCR_ERR_ARG;
  if (k < 1 || k > FTGCR_MAX_K) return FTGCR_ERR_ARG;
  if (!(tol > 0.0) || !std::isfinite(tol)) return FTGCR_ERR_ARG;
  if (g->max_steps < 0 || g->tiles < 0 || g->max_outer < 0 || !(g->inner_tol >= 0.0) || g->inner_tol >= 1.0)
    return FTGCR_ERR_ARG;
  constexpr int layouts = FTGCR_FLAG_SPLIT_ROUNDS | FTGCR_FLAG_FUSED_ROUNDS | FTGCR_FLAG_STREAMED_ROUNDS;
  if (g->flags & ~(FTGCR_FLAG_UNPROTECTED | FTGCR_FLAG_ORACLE_ORDER | FTGCR_FLAG_ZERO_GUESS | layouts))
    return FTGCR_ERR_ARG;
  if ((g->flags & FTGCR_FLAG_ORACLE_ORDER) && g->precision != FTGCR_FP64) return FTGCR_ERR_ARG;
  const int lf = g->flags & layouts;
  if (lf & (lf - 1)) return FTGCR_ERR_ARG;  // at most one layout
  if ((g->flags & (FTGCR_FLAG_SPLIT_ROUNDS | FTGCR_FLAG_STREAMED_ROUNDS)) &&
      (g->precision != FTGCR_MIXED || g->precond != FTGCR_PRECOND_LINE))
    return FTGCR_ERR_ARG;
  // mu = 0 on a single latitude row leaves the zonal line systems singular
  if (g->mu == 0.0 && g->nlat < 2 && g->precond != FTGCR_PRECOND_IDENTITY) return FTGCR_ERR_ARG;
  return FTGCR_OK;
}

static void fill_handle_params(ftgcr_handle* h, const ftgcr_grid* g, int32_t k, double tol, int sms, int smem_limit) {
  h->nlon = g->nlon;
  h->nlat = g->nlat;
  h->k = k;
  h->tol = tol;
  h->mu = g->mu;
  h->precision = g->precision;
  h->precond = g->precond;
  h->N = (long long)g->nlon * g->nlat;
  h->C = chunk_len(g->nlon);
  h->max_steps = g->max_steps > 0 ? g->max_steps : 100LL * (long long)std::ceil(std::sqrt((double)h->N)) + 100;
  h->inner_tol = g->inner_tol > 0 ? g->inner_tol : 1e-5;
  h->max_outer = g->max_outer > 0 ? g->max_outer : 40;
  h->flags = g->flags;
  const bool mixed = g->precision == FTGCR_MIXED;
  const size_t elem = mixed ? sizeof(float) : sizeof(double);
  int gconsts = 0;
  choose_tiling(g->nlon, g->nlat, mixed, elem, g->precond, g->flags, g->tiles, sms, (size_t)smem_limit, k, &h->nt,
                &h->split, &gconsts);
  if (h->split == 2) {
    stream_plan(h->nlon, k, (size_t)smem_limit, &h->plan);
    h->wide = 2;
    return;
  }
  if (h->split < 0) {  // streamed rounds asked for where they do not fit
    h->split = 0;
    h->plan.bytes = (size_t)smem_limit + 1;
    h->wide = 0;
    return;
  }
  h->plan = smem_plan(h->nlon, h->nlat, h->nt, mixed, elem, h->precond, h->split, (size_t)smem_limit, gconsts);
  h->wide = h->split || h->plan.gconsts;
}

int ftgcr_create(const ftgcr_grid* grid, const ftgcr_coeffs* coeffs, int32_t k, double tol, ftgcr_handle** out) {
  if (!out) return FTGCR_ERR_ARG;
  *out = nullptr;
  int rc = check_grid(grid, k, tol);
  if (rc) return rc;
  if (!coeffs || !coeffs->D) return FTGCR_ERR_ARG;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  const DeviceInfo di = device_info(dev);
  const int smem_limit = di.smem_optin - kStaticSmemReserve;
  ftgcr_handle* h = new ftgcr_handle();
  h->dev = dev;
  fill_handle_params(h, grid, k, tol, di.sms, smem_limit);
  const bool mixed = grid->precision == FTGCR_MIXED;
  if (h->plan.bytes > (size_t)smem_limit) {
    delete h;
    return FTGCR_ERR_ARG;  // a single latitude row does not fit on chip
  }
  const bool Ddev = is_device_ptr(coeffs->D);
  if (!Ddev) {
    for (long long i = 0; i < h->N; ++i)
      if (!std::isfinite(coeffs->D[i]) || !(coeffs->D[i] > 0.0)) {
        delete h;
        return FTGCR_ERR_ARG;
      }
  }
  rc = mixed ? create_impl<float>(h, coeffs->D, Ddev) : create_impl<double>(h, coeffs->D, Ddev);
  if (rc) {
    ftgcr_destroy(h);
    return rc;
  }
  *out = h;
  return FTGCR_OK;
}

int ftgcr_set_coeffs(ftgcr_handle* h, const ftgcr_coeffs* coeffs, void* stream) {
  if (!h || !coeffs || !coeffs->D) return FTGCR_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const bool Ddev = is_device_ptr(coeffs->D);
  const double* Dd = coeffs->D;
  double* dD = nullptr;
  if (!Ddev) {
    for (long long i = 0; i < h->N; ++i)
      if (!std::isfinite(coeffs->D[i]) || !(coeffs->D[i] > 0.0)) return FTGCR_ERR_ARG;
    CK(cudaMallocAsync((void**)&dD, sizeof(double) * h->N, st));
    CK(cudaMemcpyAsync(dD, coeffs->D, sizeof(double) * h->N, cudaMemcpyHostToDevice, st));
    Dd = dD;
  }
  const int rc = h->precision == FTGCR_MIXED ? setup_coefficients<float>(h, h->sd32, Dd, st)
                                             : setup_coefficients<double>(h, h->sd64, Dd, st);
  if (dD) cudaFreeAsync(dD, st);
  if (!Ddev) CK(cudaStreamSynchronize(st));  // the host array may be reused as soon as this returns
  return rc;
}

int64_t ftgcr_footprint(const ftgcr_grid* grid, int32_t k) {
  if (check_grid(grid, k, 1.0)) return -1;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    dev = 0;
  }
  const DeviceInfo di = device_info(dev);
  ftgcr_handle h;
  fill_handle_params(&h, grid, k, 1.0, di.sms > 0 ? di.sms : 152, di.smem_optin > 0 ? di.smem_optin - kStaticSmemReserve : 200000);
  size_t b;
  if (grid->precision == FTGCR_MIXED) {
    SolveDev<float> sd{};
    b = layout<float>(&h, nullptr, &sd);
  } else {
    SolveDev<double> sd{};
    b = layout<double>(&h, nullptr, &sd);
  }
  return (int64_t)b + 3 * (int64_t)h.N * (int64_t)sizeof(double);  // + create-time scratch
}

int ftgcr_solve_async(ftgcr_handle* h, const double* rhs, double* x, const ftgcr_fault_plan* plan, void* stream) {
  if (!h || !rhs || !x) return FTGCR_ERR_ARG;
  int rc = validate_plan(h, plan);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  return h->precision == FTGCR_MIXED ? solve_async_impl<float>(h, rhs, x, x, plan, st)
                                     : solve_async_impl<double>(h, rhs, x, x, plan, st);
}

// The work of ftgcr_solve up to the copy of the solution back, enqueued on
// the stream without waiting for it.
static int solve_enqueue(ftgcr_handle* h, const double* rhs, double* x, const ftgcr_fault_plan* plan,
                         cudaStream_t st) {
  if (!h || !rhs || !x) return FTGCR_ERR_ARG;
  int rc = validate_plan(h, plan);
  if (rc) return rc;
  const bool rdev = is_device_ptr(rhs), xdev = is_device_ptr(x);
  const double* R = rhs;
  double* X = x;
  // host arrays: staged, and checked for finite values on the device (the
  // solve does not start if one is not; x then comes back unchanged).  With
  // FTGCR_FLAG_ZERO_GUESS x is output only: not copied in nor checked (its
  // staging buffer is zeroed, which a refused solve returns)
  const bool zg = (h->flags & FTGCR_FLAG_ZERO_GUESS) != 0;
  const bool check = !rdev || (!xdev && !zg);
  const int cg = (int)std::min<long long>((h->N + 255) / 256, 1024);
  if (check) CK(cudaMemsetAsync(&h->ctl->nonfinite, 0, sizeof(int), st));
  if (!rdev) {
    CK(cudaMemcpyAsync(h->stageR, rhs, sizeof(double) * h->N, cudaMemcpyHostToDevice, st));
    k_nonfinite<<<cg, 256, 0, st>>>(h->stageR, h->N, h->ctl);
    R = h->stageR;
  }
  if (!xdev) {
    if (zg) {
      CK(cudaMemsetAsync(h->stageX, 0, sizeof(double) * h->N, st));
    } else {
      CK(cudaMemcpyAsync(h->stageX, x, sizeof(double) * h->N, cudaMemcpyHostToDevice, st));
      k_nonfinite<<<cg, 256, 0, st>>>(h->stageX, h->N, h->ctl);
    }
    X = h->stageX;
  }
  CK(cudaGetLastError());
  rc = h->precision == FTGCR_MIXED ? solve_async_impl<float>(h, R, X, X, plan, st, check)
                                   : solve_async_impl<double>(h, R, X, X, plan, st, check);
  if (rc) return rc;
  if (!xdev) CK(cudaMemcpyAsync(x, h->stageX, sizeof(double) * h->N, cudaMemcpyDeviceToHost, st));
  return FTGCR_OK;
}

int ftgcr_solve(ftgcr_handle* h, const double* rhs, double* x, const ftgcr_fault_plan* plan, void* stream) {
  cudaStream_t st = (cudaStream_t)stream;
  const int rc = solve_enqueue(h, rhs, x, plan, st);
  if (rc) return rc;
  CK(cudaStreamSynchronize(st));
  h->last_status = status_from_result(h);
  trace_dump(h->grid);
  return h->last_status;
}

int ftgcr_solve_host_async(ftgcr_handle* h, const double* rhs, double* x, const ftgcr_fault_plan* plan,
                           void* stream) {
  return solve_enqueue(h, rhs, x, plan, (cudaStream_t)stream);
}

int ftgcr_stats(ftgcr_handle* h, ftgcr_stats_t* out) {
  if (!h || !out) return FTGCR_ERR_ARG;
  if (!h->solved) return FTGCR_ERR_STATE;
  CK(cudaStreamSynchronize(h->last_stream));
  h->last_status = status_from_result(h);
  const SolveState& S = *h->h_result;
  memset(out, 0, sizeof *out);
  out->steps = S.step;
  out->cycles = S.cycles;
  out->restarts = S.restarts;
  out->faults_injected = S.finj;
  out->faults_detected = S.fdet;
  out->outer = h->precision == FTGCR_MIXED ? std::max(0, S.outer - 1) : 0;
  out->ndetect = S.ndetect;
  out->converged = S.status == ST_CONVERGED;
  for (int q = 0; q < S.ndetect && q < FTGCR_MAX_DETECT; ++q) {
    out->detect_step[q] = S.detect_step[q];
    out->detect_ratio[q] = S.detect_ratio[q];
  }
  out->res0 = std::sqrt(S.nrm2_0);
  out->res_final_rec = std::sqrt(S.nrm2_last);
  out->res_final_true = std::sqrt(S.res_true2);
  out->norm_R = std::sqrt(S.nrm2_R);
  out->bytes_resident = (int64_t)h->pool_bytes;
  out->bytes_backup = (int64_t)h->backup_bytes;
  out->tiles = h->nt;
  out->status = h->last_status;
  out->loss_events = S.lossev;
  out->split_rounds = h->split;
  out->global_factors = h->plan.gconsts;
  return FTGCR_OK;
}

int ftgcr_apply_operator(ftgcr_handle* h, const double* in, double* out, void* stream) {
  if (!h || !in || !out) return FTGCR_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = (int)std::min<long long>((h->N + 255) / 256, 4096);
  k_apply_operator<<<blocks, 256, 0, st>>>(in, out, h->Tx64, h->Ty64, h->muA64, h->nlon, h->nlat);
  CK(cudaGetLastError());
  return FTGCR_OK;
}

int ftgcr_apply_precond(ftgcr_handle* h, const double* in, double* out, void* stream) {
  if (!h || !in || !out) return FTGCR_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  SolveDev<double> sd{};
  if (h->precision == FTGCR_FP64) {
    sd = h->sd64;
  } else {
    return FTGCR_ERR_ARG;  // the FP64 factorisation is only kept by FP64 handles
  }
  const int rows_per_block = 4;
  const size_t smem = (size_t)rows_per_block * row_stride(h->nlon) * sizeof(double);
  CK(cudaFuncSetAttribute(k_apply_precond, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_apply_precond<<<(h->nlat + rows_per_block - 1) / rows_per_block, 32 * rows_per_block, smem, st>>>(in, out, sd);
  CK(cudaGetLastError());
  return FTGCR_OK;
}

int ftgcr_solve_batch(ftgcr_handle* const* hs, const double* const* rhs, double* const* x,
                      const ftgcr_fault_plan* const* plans, int32_t n, void* stream) {
  if (!hs || !rhs || !x || n < 1 || n > kMaxBatch) return FTGCR_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (!hs[i] || !rhs[i] || !x[i] || hs[i]->precision != hs[0]->precision || hs[i]->dev != hs[0]->dev)
      return FTGCR_ERR_ARG;
    for (int j = 0; j < i; ++j)
      if (hs[j] == hs[i]) return FTGCR_ERR_ARG;  // one solve per handle per launch
    const int rc = validate_plan(hs[i], plans ? plans[i] : nullptr);
    if (rc) return rc;
  }
  cudaStream_t st = (cudaStream_t)stream;
  return hs[0]->precision == FTGCR_MIXED ? solve_batch_impl<float>(hs, rhs, x, plans, n, st)
                                         : solve_batch_impl<double>(hs, rhs, x, plans, n, st);
}

void ftgcr_destroy(ftgcr_handle* h) {
  if (!h) return;
  if (h->pool) cudaFree(h->pool);
  if (h->h_result) cudaFreeHost(h->h_result);
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  delete h;
}

}  // extern "C"

// ------------------------------------------------------------ slot tables (scheduler interface)
namespace ftgcr {
namespace serve {

struct SlotTable : SlotTableImpl {};

int table_create(int precision, int max_slots, SlotTable** out) {
  if (!out || max_slots < 1 || max_slots > 1024 || (precision != FTGCR_FP64 && precision != FTGCR_MIXED))
    return FTGCR_ERR_ARG;
  SlotTable* t = new SlotTable();
  t->precision = precision;
  t->n = max_slots;
  t->slot.assign(max_slots, nullptr);
  t->launched.assign(max_slots, 0);
  CK(cudaGetDevice(&t->dev));
  const DeviceInfo di = device_info(t->dev);
  t->grid_cap = di.sms * 4;
  const size_t b_solves = align256(sizeof(void*) * max_slots), b_nt = align256(sizeof(int) * max_slots),
               b_act = align256(sizeof(int) * 2 * max_slots), b_ctl = align256(sizeof(LaunchCtl)),
               b_diag = align256(sizeof(int) * 4 * t->grid_cap), b_res = align256(sizeof(SolveState) * max_slots);
  const size_t total = b_solves + b_nt + b_act + b_ctl + b_diag + b_res;
  if (cudaMalloc(&t->buf, total) != cudaSuccess) {
    cudaGetLastError();
    delete t;
    return FTGCR_ERR_OOM;
  }
  t->d_solves = (void**)t->buf;
  t->d_nt = (int*)(t->buf + b_solves);
  t->d_act = (int*)(t->buf + b_solves + b_nt);
  t->d_ctl = (LaunchCtl*)(t->buf + b_solves + b_nt + b_act);
  t->d_diag = (int*)(t->buf + b_solves + b_nt + b_act + b_ctl);
  t->d_results = (SolveState*)(t->buf + b_solves + b_nt + b_act + b_ctl + b_diag);
  int rc = cuda_status(cudaMemset(t->buf, 0, total));
  if (!rc) rc = cuda_status(cudaMallocHost(&t->h_ctl_in, sizeof(LaunchCtl)));
  if (!rc) rc = cuda_status(cudaMallocHost(&t->h_ctl_out, sizeof(LaunchCtl)));
  if (!rc) rc = cuda_status(cudaMallocHost(&t->h_act, sizeof(int) * 2 * max_slots));
  if (!rc) rc = cuda_status(cudaMallocHost(&t->h_results, sizeof(SolveState) * max_slots));
  if (rc) {
    table_destroy(t);
    return rc;
  }
  *out = t;
  return FTGCR_OK;
}

void table_destroy(SlotTable* t) {
  if (!t) return;
  if (t->buf) cudaFree(t->buf);
  if (t->h_ctl_in) cudaFreeHost(t->h_ctl_in);
  if (t->h_ctl_out) cudaFreeHost(t->h_ctl_out);
  if (t->h_act) cudaFreeHost(t->h_act);
  if (t->h_results) cudaFreeHost(t->h_results);
  delete t;
}

__global__ void k_table_place(void** solves, int* nt, int slot, void* sdev, int tiles) {
  solves[slot] = sdev;
  nt[slot] = tiles;
}

int table_begin(SlotTable* t, int slot, ftgcr_handle* h, const double* rhs, double* x, const ftgcr_fault_plan* plan,
                cudaStream_t st, int check) {
  if (!t || !h || !rhs || !x || slot < 0 || slot >= t->n || t->slot[slot] || h->precision != t->precision)
    return FTGCR_ERR_ARG;
  for (ftgcr_handle* o : t->slot)
    if (o == h) return FTGCR_ERR_ARG;  // one running solve per handle
  int rc = validate_plan(h, plan);
  if (rc) return rc;
  // written by a kernel, not copied from pageable host memory: such a copy
  // may wait for the launch still running on the stream
  k_table_place<<<1, 1, 0, st>>>(t->d_solves, t->d_nt, slot, h->sdev, h->nt);
  CK(cudaGetLastError());
  if (check) {  // the handle's own control block carries the flag
    const int cg = (int)std::min<long long>((h->N + 255) / 256, 1024);
    CK(cudaMemsetAsync(&h->ctl->nonfinite, 0, sizeof(int), st));
    if (check & 1) k_nonfinite<<<cg, 256, 0, st>>>(rhs, h->N, h->ctl);
    if (check & 2) k_nonfinite<<<cg, 256, 0, st>>>(x, h->N, h->ctl);
  }
  const BeginArgs b = begin_args(h, rhs, x, x, plan);
  // parity -1: the begin may be enqueued behind a launch still running
  const LaunchCtl* chk = check ? h->ctl : nullptr;
  if (t->precision == FTGCR_MIXED)
    k_begin_solve<float><<<1, 64, 0, st>>>((SolveDev<float>*)h->sdev, b, t->d_act, t->n, slot, -1, nullptr, chk);
  else
    k_begin_solve<double><<<1, 64, 0, st>>>((SolveDev<double>*)h->sdev, b, t->d_act, t->n, slot, -1, nullptr, chk);
  CK(cudaGetLastError());
  t->slot[slot] = h;
  return FTGCR_OK;
}

int table_run(SlotTable* t, int max_rounds, cudaStream_t st) {
  if (!t || max_rounds < 1) return FTGCR_ERR_ARG;
  return t->precision == FTGCR_MIXED ? table_run_impl<float>(t, max_rounds, st)
                                     : table_run_impl<double>(t, max_rounds, st);
}

int table_collect(SlotTable* t, cudaStream_t st, int* finished) {
  if (!t || !finished) return FTGCR_ERR_ARG;
  for (int s = 0; s < t->n; ++s) finished[s] = 0;
  bool any = false;
  for (int s = 0; s < t->n; ++s) any = any || (t->launched[s] && t->slot[s]);
  if (!any) return FTGCR_OK;
  CK(cudaStreamSynchronize(st));
  const int err = t->h_ctl_out->err;
  t->round = t->h_ctl_out->round_end;
  const int par = (int)(t->round & 1);
  for (int s = 0; s < t->n; ++s) {
    ftgcr_handle* h = t->slot[s];
    if (!h || !t->launched[s]) continue;  // begun after the launch: runs in the next one
    t->launched[s] = 0;
    if (!err && t->h_act[par * t->n + s]) continue;
    memcpy(h->h_result, t->h_results + s, sizeof(SolveState));  // gathered after the launch
    *h->h_ctl = *t->h_ctl_out;
    h->last_stream = st;
    h->solved = 1;
    h->last_status = err ? FTGCR_ERR_TIMEOUT : status_from_result(h);
    finished[s] = 1;
    t->slot[s] = nullptr;
  }
  if (err) {
    // the launch is abandoned: its solves' state is not resumable, and the
    // next launch starts from a clean table
    CK(cudaMemsetAsync(t->d_act, 0, sizeof(int) * 2 * t->n, st));
    CK(cudaStreamSynchronize(st));
    return FTGCR_ERR_TIMEOUT;
  }
  return FTGCR_OK;
}

void table_abandon(SlotTable* t, cudaStream_t st) {
  for (auto& h : t->slot) h = nullptr;
  cudaMemsetAsync(t->d_act, 0, sizeof(int) * 2 * t->n, st);
  cudaStreamSynchronize(st);
}

int table_occupied(const SlotTable* t) {
  int n = 0;
  for (ftgcr_handle* h : t->slot) n += h != nullptr;
  return n;
}
int table_slots(const SlotTable* t) { return t->n; }

double* handle_stage_rhs(ftgcr_handle* h) { return h->stageR; }
double* handle_stage_x(ftgcr_handle* h) { return h->stageX; }
long long handle_points(const ftgcr_handle* h) { return h->N; }
int handle_precision(const ftgcr_handle* h) { return h->precision; }

}  // namespace serve
}  // namespace ftgcr

// ------------------------------------------------------------ no-allocation solve
// Some callers cannot allocate device memory when they solve: processes whose
// device memory is owned entirely by another allocator (a framework's caching
// pool, an arena reserved at start-up), and code that must not fail with
// out-of-memory in the middle of a run.  For them, ftgcr_solve_noalloc keeps
// all of its scratch in the static device array below instead of allocating a
// handle's pool.  Every GPU that loads the library holds the array until the
// process exits.  The call blocks (it stages small records through host
// memory and synchronises its stream), so it is not meant for stream capture.
constexpr long long kNoAllocMaxPoints = FTGCR_NOALLOC_MAX_POINTS;
constexpr int kNoAllocMaxK = FTGCR_NOALLOC_MAX_K;
static __device__ __align__(256) unsigned char g_noalloc_scratch[FTGCR_NOALLOC_SCRATCH_BYTES];

namespace {

struct NoAllocDevice {
  unsigned char* base = nullptr;  // device address of g_noalloc_scratch
  bool ready = false;
};

// Set-up, once per device, with that device current: the device address of
// the static array (in host code its name is only a host-side stand-in).
int noalloc_base(int dev, unsigned char** base) {
  static std::mutex mu;
  static std::vector<NoAllocDevice> devs;
  std::lock_guard<std::mutex> lk(mu);
  if ((int)devs.size() <= dev) devs.resize(dev + 1);
  if (!devs[dev].ready) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return FTGCR_ERR_CUDA;
    }
    devs[dev].base = (unsigned char*)p;
    devs[dev].ready = true;
  }
  *base = devs[dev].base;
  return FTGCR_OK;
}

}  // namespace

extern "C" int ftgcr_solve_noalloc(const ftgcr_grid* grid, const double* D, int32_t k, double tol, const double* rhs,
                                   double* x, ftgcr_stats_t* stats, void* stream) {
  int rc = check_grid(grid, k, tol);
  if (rc) return rc;
  if (!D || !rhs || !x || grid->precision != FTGCR_FP64 || grid->precond != FTGCR_PRECOND_LINE)
    return FTGCR_ERR_ARG;
  if ((long long)grid->nlon * grid->nlat > kNoAllocMaxPoints || k > kNoAllocMaxK) return FTGCR_ERR_ARG;
  if (!is_device_ptr(D) || !is_device_ptr(rhs) || !is_device_ptr(x)) return FTGCR_ERR_ARG;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  unsigned char* base = nullptr;
  rc = noalloc_base(dev, &base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const DeviceInfo di = device_info(dev);
  const int smem_limit = di.smem_optin - kStaticSmemReserve;

  // the handle record lives on the host stack; its pool is the static array
  ftgcr_handle h;
  h.dev = dev;
  h.noalloc = 1;  // the serial row solve: no chunk-layout factors in the fixed scratch
  fill_handle_params(&h, grid, k, tol, di.sms, smem_limit);
  if (h.plan.bytes > (size_t)smem_limit) return FTGCR_ERR_ARG;
  SolveDev<double> sd{};
  const size_t pool = layout<double>(&h, nullptr, &sd);
  const size_t geo = align256(sizeof(double) * 3 * h.nlat);
  if (pool + geo > (size_t)FTGCR_NOALLOC_SCRATCH_BYTES) return FTGCR_ERR_ARG;
  layout<double>(&h, base, &sd);
  double* dgeo = (double*)(base + pool);

  sd.nlon = h.nlon;
  sd.nlat = h.nlat;
  sd.k = h.k;
  sd.nt = h.nt;
  sd.nt_hmax = (h.nlat + h.nt - 1) / h.nt;
  sd.C = h.C;
  sd.precond = h.precond;
  sd.mixed = 0;
  sd.N = h.N;
  sd.max_steps = h.max_steps;
  sd.max_outer = h.max_outer;
  sd.tol2 = h.tol * h.tol;
  sd.inner_tol2 = h.inner_tol * h.inner_tol;
  sd.protect = (h.flags & FTGCR_FLAG_UNPROTECTED) ? 0 : 1;
  sd.zero_guess = (h.flags & FTGCR_FLAG_ZERO_GUESS) ? 1 : 0;
  sd.oracle_order = (h.flags & FTGCR_FLAG_ORACLE_ORDER) ? 1 : 0;
  sd.split = 0;
  sd.cs_off = (int)h.plan.cs_off;
  sd.cs_clobber = 0;
  sd.cs_global = h.plan.gconsts;
  sd.Tx64 = h.Tx64;
  sd.Ty64 = h.Ty64;
  sd.muA64 = h.muA64;

  // The array keeps the last call's contents, laid out for that call's sizes:
  // clear the part this call uses, so that it starts from the state of a
  // freshly created handle, then write the coefficients and factorisation.
  CK(cudaMemsetAsync(base, 0, pool + geo, st));
  std::vector<double> cx, cy, area, g3;
  row_geometry(h.nlon, h.nlat, cx, cy, area);
  g3.insert(g3.end(), cx.begin(), cx.end());
  g3.insert(g3.end(), cy.begin(), cy.end());
  g3.insert(g3.end(), area.begin(), area.end());
  CK(cudaMemcpyAsync(dgeo, g3.data(), sizeof(double) * 3 * h.nlat, cudaMemcpyHostToDevice, st));
  k_face_coeffs<<<256, 256, 0, st>>>(h.nlon, h.nlat, D, dgeo, dgeo + h.nlat, dgeo + 2 * h.nlat, h.mu, h.Tx64, h.Ty64,
                                     h.muA64, nullptr, nullptr, nullptr);
  CK(cudaGetLastError());
  rc = launch_line_factor(h.nlon, h.nlat, h.C, h.precond, h.Tx64, h.Ty64, h.muA64, (double*)sd.lc, (double*)sd.lw,
                          (double*)sd.lu, (double*)sd.lz, (double*)sd.lrow, nullptr, nullptr, nullptr, nullptr, st);
  if (rc) return rc;
  void* sp = h.sdev;
  CK(cudaMemcpyAsync(h.sdev, &sd, sizeof sd, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h.sdev_arr, &sp, sizeof(void*), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(h.nt_dev, &h.nt, sizeof(int), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(h.active, 0, sizeof(int) * 2, st));

  const int kb = kbound(h.k);
  h.smem = h.plan.bytes;
  rc = configure_kernel<double>(kb, h.wide, std::max<size_t>(h.smem, 1));
  if (rc) return rc;
  int occ = 0;
  rc = occupancy<double>(kb, h.wide, h.smem, &occ);
  if (rc) return rc;
  if (occ < 1) return FTGCR_ERR_ARG;
  {
    // no stack resize here (it may allocate): the current limit must cover
    // the kernel's frame with the margin ftgcr_create keeps
    cudaFuncAttributes fa;
    CK(cudaFuncGetAttributes(&fa, kernel_ptr<double>(kb, h.wide)));
    size_t cur = 0;
    CK(cudaDeviceGetLimit(&cur, cudaLimitStackSize));
    if (fa.localSizeBytes + 256 > cur) return FTGCR_ERR_ARG;
  }
  const int grid_ctas = std::min(h.nt, di.sms * occ);
  const BeginArgs b = begin_args(&h, rhs, x, x, nullptr);
  k_begin_solve<double><<<1, 64, 0, st>>>((SolveDev<double>*)h.sdev, b, h.active, 1, 0, 0, h.ctl);
  CK(cudaGetLastError());
  BatchArgs<double> a;
  a.solves = (SolveDev<double>* const*)h.sdev_arr;
  a.nt = h.nt_dev;
  a.active = h.active;
  a.n = 1;
  a.ctl = h.ctl;
  a.max_rounds = (int)std::min<long long>(1 << 30, 2 * h.max_steps + 8 * ((long long)h.max_outer + 2) + 16);
  a.trace = nullptr;
  a.trace_rounds = 0;
  a.diag = h.diag;
  void* args[] = {&a};
  CK(cudaLaunchCooperativeKernel(kernel_ptr<double>(kb, h.wide), dim3(grid_ctas), dim3(kThreads), args, h.smem, st));
  SolveState res;
  LaunchCtl ctl;
  CK(cudaMemcpyAsync(&res, h.result, sizeof res, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&ctl, h.ctl, sizeof ctl, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  int status = ctl.err ? FTGCR_ERR_TIMEOUT
                       : (res.active ? FTGCR_ERR_CUDA : (res.status == ST_CONVERGED ? FTGCR_OK : FTGCR_NOT_CONVERGED));
  if (stats) {
    memset(stats, 0, sizeof *stats);
    stats->steps = res.step;
    stats->cycles = res.cycles;
    stats->restarts = res.restarts;
    stats->faults_injected = res.finj;
    stats->faults_detected = res.fdet;
    stats->ndetect = res.ndetect;
    stats->converged = res.status == ST_CONVERGED;
    for (int q = 0; q < res.ndetect && q < FTGCR_MAX_DETECT; ++q) {
      stats->detect_step[q] = res.detect_step[q];
      stats->detect_ratio[q] = res.detect_ratio[q];
    }
    stats->res0 = std::sqrt(res.nrm2_0);
    stats->res_final_rec = std::sqrt(res.nrm2_last);
    stats->res_final_true = std::sqrt(res.res_true2);
    stats->norm_R = std::sqrt(res.nrm2_R);
    stats->bytes_resident = (int64_t)FTGCR_NOALLOC_SCRATCH_BYTES;
    stats->bytes_backup = (int64_t)h.backup_bytes;
    stats->tiles = h.nt;
    stats->status = status;
  }
  // the host record must not free anything: nothing was allocated
  h.pool = nullptr;
  h.h_result = nullptr;
  h.h_ctl = nullptr;
  return status;
}

