// Device-side building blocks of the FT-GCR(k) library: solve descriptors, the
// per-solve state machine record, reductions, the bounded grid barrier, the
// finite-volume stencil (Eq. (1) operator) and the zonal line solve
// (preconditioner e = P^-1(r) of Algorithm 1).
//
// Compiled with --fmad=false: every multiply-add that the method fuses is an
// explicit fma()/fmaf(); everything else is rounded operation by operation.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ftgcr {

constexpr int kMaxK = 16;
constexpr int kNSlot = kMaxK + 2;      // p / L(p) buffers
constexpr int kMaxFaults = 64;
constexpr int kMaxDetect = 16;
constexpr int kNPart = kMaxK + 2;      // partial sums per tile
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned long long kBarrierTimeoutNs = 2000000000ull;  // 2 s
constexpr unsigned long long kKernelTimeoutNs = 60000000000ull;  // 60 s

// Phase kinds of the persistent state machine.
enum Kind : int {
  K_NONE = 0,     // nothing pending (fresh solve) / no work this round
  K_INIT = 1,     // r0 = L(phi0) - R, p0 = P^-1 r0, L(p0), first dots
  K_PA = 2,       // axpy + ||r||^2 + e = P^-1 r + L(e) + <L(e), L(p^l)>
  K_PB = 3,       // p^{nu+1}, L(p^{nu+1}) recurrences + next-beta dots
  K_RESTORE = 4,  // [phi, r, p, L(p)]^0 <- ^* after a detected fault
  K_OUT = 5,      // mixed: x += d, r_out = R - L64(x), inner right-hand side
  K_FIN = 6       // write x, true residual
};
enum Vec : int { V_X = 0, V_R = 1, V_P = 2, V_AP = 3, V_E = 4 };
enum Precond : int { PC_LINE = 0, PC_JACOBI = 1, PC_IDENTITY = 2 };
enum Status : int { ST_RUNNING = 0, ST_CONVERGED = 1, ST_NOT_CONVERGED = 2 };

struct Fault {  // same layout as ftgcr_fault
  long long step;
  int vec;
  long long index;
  int bit;
};

// Record of one solve, double-buffered by round parity.  Written by the CTA
// that owns tile 0 of the solve, read by every CTA that works on the solve in
// the next round.  Every CTA recomputes the same transition from it.
struct SolveState {
  int active;
  int pending;  // phase whose partial sums wait in the partials buffer
  int nu;
  int outer;
  long long step;  // executed steps so far
  int phiC, phiW, phiS, rC, rW, rS;
  int slot[kMaxK + 1];
  int slotS;
  int patched;  // the backup still carries the clean values of the init flips
  long long patch_step;  // step of those flips
  int xcur;     // mixed: x ping-pong buffer holding the current x
  int finbuf;   // phi buffer of the final iterate (FIN) / inner solution (OUT)
  int finzero;  // FIN writes x = 0 (R = 0)
  int first_out;
  int stag;     // mixed: detections since the last accepted step
  int status;
  double beta;
  double lpn2[kMaxK + 1];
  double nrm2_prev, nrm2_S, nrm2_R, thr2, nrm2_0, nrm2_last, nrm2_out, thr2_in, res_true2;
  long long cycles, restarts, finj, fdet;
  int ndetect, pad;
  long long detect_step[kMaxDetect];
  double detect_ratio[kMaxDetect];
};

// Static description of one solve (pointers into the handle's allocations).
template <typename T>
struct SolveDev {
  int nlon, nlat, k, nt, C, precond, mixed, nfaults;
  long long N, max_steps;
  int max_outer;
  double tol2, inner_tol2;
  // operator (inner precision)
  const T* Tx;
  const T* Ty;
  const T* muA;   // [nlat]
  // preconditioner: line solve constants permuted [nlat][C][32]; jacobi: 1/diag natural
  const T* lc;
  const T* lw;
  const T* lz;
  const T* lrow;  // [nlat][4]: 1/delta, Tx_{n-1}/delta, Tx_{n-2}/delta, 0
  // Krylov vectors (inner precision)
  T* phi[3];
  T* r[3];
  T* e;
  T* Le;
  T* p[kNSlot];
  T* Lp[kNSlot];
  T* Rin;          // mixed: FP32 inner right-hand side
  // FP64 operator and outer vectors
  const double* Tx64;
  const double* Ty64;
  const double* muA64;
  double* xbuf[2];  // mixed: x ping-pong
  const double* R;  // user right-hand side (device)
  const double* x0; // user initial guess (device)
  double* xout;     // user solution (device)
  // bookkeeping
  double* part;      // [2][nt][kNPart]
  SolveState* st;    // [2]
  SolveState* result;  // final record (written once)
  const Fault* faults;
  double* patchval;  // [kMaxFaults]
};

// --------------------------------------------------------------- helpers
__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldcg(const float* p) { return __ldcg(p); }

__device__ __forceinline__ double flip_bits(double v, int bit) {
  unsigned long long u = __double_as_longlong(v);
  u ^= 1ull << (bit & 63);
  return __longlong_as_double(u);
}
__device__ __forceinline__ float flip_bits(float v, int bit) {
  unsigned int u = __float_as_uint(v);
  u ^= 1u << (bit & 31);
  return __uint_as_float(u);
}

__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }

// Inner-product accumulator.  FP64 vectors: one fma per element.  FP32
// vectors: the product of two floats is formed exactly as a float pair
// (TwoProd) and accumulated in a float-float pair (TwoSum); the pair is
// promoted to FP64 once per thread, and all further reduction is FP64.
template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double s;
  __device__ __forceinline__ Acc() : s(0.0) {}
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ double get() const { return s; }
};
template <>
struct Acc<float> {
  float hi, lo;
  __device__ __forceinline__ Acc() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ void add(float a, float b) {
    float p = a * b;
    float pe = fmaf(a, b, -p);
    float s = hi + p;
    float bb = s - hi;
    float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo = lo + (err + pe);
  }
  __device__ __forceinline__ double get() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Deterministic CTA reduction of nv per-thread values; the sums land in
// out[0..nv-1] (global).  red_smem: kWarps * kNPart doubles.
__device__ __forceinline__ void cta_reduce_store(const double* vals, int nv, double* red_smem, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int v = 0; v < nv; ++v) {
    double s = warp_sum(vals[v]);
    if (lane == 0) red_smem[warp * kNPart + v] = s;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += red_smem[w * kNPart + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier for a cooperative launch: monotonic arrival counter (zeroed
// before the launch), bounded spin.  On timeout the CTA raises *err and
// returns; every CTA checks *err after each barrier, so the kernel ends
// within one more timeout.  Returns false when the kernel must stop.
__device__ __forceinline__ bool grid_barrier(unsigned int* counter, unsigned int target, int* err, int* bail_smem) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(counter, 1u);
    unsigned long long t0 = globaltimer();
    unsigned int it = 0;
    while (ld_acquire_u32(counter) < target) {
      if ((++it & 63u) == 0u && globaltimer() - t0 > kBarrierTimeoutNs) {
        atomicExch(err, 1);
        break;
      }
      __nanosleep(40);
    }
    __threadfence();
    *bail_smem = *(volatile int*)err;
  }
  __syncthreads();
  return *bail_smem == 0;
}

// --------------------------------------------------------------- operator
// (L v)_{j,i} of Eq. (1), identical operation order to the CPU oracle:
// Tx_c (v_E - v) + Tx_W (v_W - v) [+ Ty_c (v_N - v)] [+ Ty_S (v_S - v)] - muA v
template <typename T>
__device__ __forceinline__ T stencil5(T v, T ve, T vw, T vn, T vs, T txc, T txw, T tyc, T tys, T muA, bool hasN,
                                      bool hasS) {
  T s = txc * (ve - v) + txw * (vw - v);
  if (hasN) s = s + tyc * (vn - v);
  if (hasS) s = s + tys * (vs - v);
  return s - muA * v;
}

// Shared-memory row layout: element i of a row lives at i + i/32 (one pad
// word per 32), which keeps both the coalesced sweeps and the per-lane
// contiguous chunks of the line solve free of bank conflicts.
__host__ __device__ __forceinline__ int sk(int i) { return i + (i >> 5); }
__host__ __device__ __forceinline__ int row_stride(int nlon) {
  int s = nlon + (nlon >> 5) + 1;
  return (s + 3) & ~3;
}

// ----------------------------------------------------------- line solve
// Periodic tridiagonal solve of one latitude row, M e = -r (P = -M is the
// zonal part of L plus the diagonal of the rest), in place in shared memory,
// by one warp.  Leading (n-1) x (n-1) block by a precomputed LU factorisation
// (c_i = Tx_i / w_i, winv_i = 1 / w_i), its two first-order recurrences run
// as 32 contiguous per-lane chunks joined by warp scans of affine maps; the
// periodic coupling of the last unknown by bordering with the precomputed
// z = A0^-1 (-Tx_{n-1} e_0 - Tx_{n-2} e_{n-2}).
template <typename T>
__device__ void line_solve_row(const SolveDev<T>& sd, int j, T* row) {
  const int lane = threadIdx.x & 31;
  const int n = sd.nlon, m = n - 1, C = sd.C;
  const T* cb = sd.lc + (long long)j * 32 * C;
  const T* cw = sd.lw + (long long)j * 32 * C;
  const T* cz = sd.lz + (long long)j * 32 * C;
  const int i0 = lane * C;
  int len = m - i0;
  len = len < 0 ? 0 : (len > C ? C : len);

  // forward: g_i = b_i + c_{i-1} g_{i-1}, b = -r
  T mylast = (len > 0) ? __ldg(cb + (len - 1) * 32 + lane) : T(0);
  T a = __shfl_up_sync(0xffffffffu, mylast, 1);
  if (lane == 0) a = T(0);
  const T a0 = a;
  T g = T(0), F = T(1);
  for (int k = 0; k < len; ++k) {
    const int s = sk(i0 + k);
    g = tfma(a, g, -row[s]);
    F = F * a;
    row[s] = g;
    a = __ldg(cb + k * 32 + lane);
  }
  T Fs = F, Gs = g;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T Fo = __shfl_up_sync(0xffffffffu, Fs, d);
    T Go = __shfl_up_sync(0xffffffffu, Gs, d);
    if (lane >= d) {
      Gs = tfma(Fs, Go, Gs);
      Fs = Fs * Fo;
    }
  }
  T carry = __shfl_up_sync(0xffffffffu, Gs, 1);
  if (lane == 0) carry = T(0);
  {
    T P = T(1);
    a = a0;
    for (int k = 0; k < len; ++k) {
      const int s = sk(i0 + k);
      P = P * a;
      row[s] = tfma(P, carry, row[s]);
      a = __ldg(cb + k * 32 + lane);
    }
  }
  // backward: y_i = winv_i g_i + c_i y_{i+1}  (c_{m-1} stored as 0)
  T y = T(0), Fb = T(1);
  for (int k = len - 1; k >= 0; --k) {
    const int s = sk(i0 + k);
    const T cc = __ldg(cb + k * 32 + lane);
    y = tfma(cc, y, row[s] * __ldg(cw + k * 32 + lane));
    Fb = Fb * cc;
    row[s] = y;
  }
  T Fr = Fb, Yr = y;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    T Fo = __shfl_down_sync(0xffffffffu, Fr, d);
    T Yo = __shfl_down_sync(0xffffffffu, Yr, d);
    if (lane + d < 32) {
      Yr = tfma(Fr, Yo, Yr);
      Fr = Fr * Fo;
    }
  }
  T carryb = __shfl_down_sync(0xffffffffu, Yr, 1);
  if (lane == 31) carryb = T(0);
  {
    T P = T(1);
    for (int k = len - 1; k >= 0; --k) {
      const int s = sk(i0 + k);
      P = P * __ldg(cb + k * 32 + lane);
      row[s] = tfma(P, carryb, row[s]);
    }
  }
  __syncwarp();
  // bordering: x_{n-1} = (b_{n-1} + Tx_{n-1} y_0 + Tx_{n-2} y_{m-1}) / delta
  const T* lr = sd.lrow + (long long)j * 4;
  const T y0 = row[sk(0)];
  const T ym = row[sk(m - 1)];
  const T bl = -row[sk(n - 1)];
  const T xl = tfma(__ldg(lr + 2), ym, tfma(__ldg(lr + 1), y0, bl * __ldg(lr + 0)));
  __syncwarp();
  for (int k = 0; k < len; ++k) {
    const int s = sk(i0 + k);
    row[s] = tfma(-xl, __ldg(cz + k * 32 + lane), row[s]);
  }
  if (lane == 0) row[sk(n - 1)] = xl;
  __syncwarp();
}

// Pointwise preconditioners on a shared-memory row (one warp).
template <typename T>
__device__ void pointwise_precond_row(const SolveDev<T>& sd, int j, T* row) {
  const int lane = threadIdx.x & 31;
  if (sd.precond == PC_JACOBI) {
    const T* dinv = sd.lw + (long long)j * sd.nlon;
    for (int i = lane; i < sd.nlon; i += 32) row[sk(i)] = -row[sk(i)] * __ldg(dinv + i);
  }
  __syncwarp();
}

template <typename T>
__device__ __forceinline__ void precond_row(const SolveDev<T>& sd, int j, T* row) {
  if (sd.precond == PC_LINE)
    line_solve_row(sd, j, row);
  else
    pointwise_precond_row(sd, j, row);
}

// Tile geometry: tile tau of nt covers rows [row_start(tau), row_start(tau+1))
// for the row phases and elements [elem_start(tau), elem_start(tau+1)) for the
// pointwise phases.  Both depend only on the solve's own sizes.
__device__ __forceinline__ int row_start(int nlat, int nt, int tau) {
  int base = nlat / nt, extra = nlat % nt;
  return tau * base + (tau < extra ? tau : extra);
}
__device__ __forceinline__ long long elem_start(long long N, int nt, int tau) {
  // multiples of 4 elements so that vector accesses stay aligned
  long long q = N >> 2;
  long long base = q / nt, extra = q % nt;
  long long s = 4 * (tau * base + (tau < extra ? tau : extra));
  return tau == nt ? N : s;
}

}  // namespace ftgcr
