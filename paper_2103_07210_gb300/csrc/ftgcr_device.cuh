// Device-side building blocks of the FT-GCR(k) library: solve descriptors, the
// per-solve state machine record, reductions, the bounded grid barrier, the
// finite-volume stencil (Eq. (1) operator) and the zonal line solve
// (preconditioner e = P^-1(r) of Algorithm 1).
//
// Compiled with --fmad=false: every multiply-add that the method fuses is an
// explicit fma()/fmaf(); everything else is rounded operation by operation.
#pragma once
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <cuda_runtime.h>

namespace ftgcr {

constexpr int kMaxK = 16;
constexpr int kNSlot = kMaxK + 2;      // p / L(p) buffers
constexpr int kMaxFaults = 64;
constexpr int kMaxDetect = 16;
constexpr int kNPart = kMaxK + 4;      // partial sums per tile (each a double-double pair)
constexpr int kPartStride = 2 * kNPart;  // doubles per tile in the partials buffer
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
  K_FIN = 6,      // write x, true residual
  K_PF = 7        // mixed: the recurrences of the previous step fused with PA
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

// Data-loss event of Section 3 (same layout as ftgcr_loss): at step `step`
// `count` entries of e in block `rank` of `nranks` each get one bit flip.
struct LossEv {
  long long step;
  int rank, nranks;
  long long count;
  unsigned long long seed;
};
constexpr int kMaxLosses = 16;

// Output i (i >= 1) of SplitMix64 started at state `seed` (Steele, Lea and
// Flood 2014): the state advances by the golden-ratio increment per output,
// each output is the state through the generator's finaliser.
__host__ __device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long i) {
  unsigned long long z = seed + i * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

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
  int xzero;    // mixed: x is zero and in no buffer yet (a zero-guess solve before its first OUT)
  int stag;     // mixed: detections since the last accepted step
  int out_redo; // mixed: this OUT recomputes r_out for the kept x (no test)
  int out_rej;  // mixed: consecutive rejected refinement updates
  int status;
  double beta;
  double lpn2[kMaxK + 1];
  double nrm2_prev, nrm2_S, nrm2_R, thr2, nrm2_0, nrm2_last, nrm2_out, thr2_in, res_true2;
  long long cycles, restarts, finj, fdet, lossev;
  int ndetect;
  int ecur;  // buffer of e, L(e) written by the latest PA / PF
  int refused;  // the solve did not start: a staged host input was not finite
  long long detect_step[kMaxDetect];
  double detect_ratio[kMaxDetect];
};

// Static description of one solve (pointers into the handle's allocations).
template <typename T>
struct SolveDev {
  int nlon, nlat, k, nt, C, precond, mixed, nfaults;
  int zero_guess;  // every solve starts from x = 0 (x not read)
  int nt_hmax;  // rows of the tallest row tile
  long long N, max_steps;
  int max_outer;
  int oracle_order;  // FP64: Dot2 sums and the oracle's stencil form (else fma forms)
  double tol2, inner_tol2;
  // operator (inner precision)
  const T* Tx;
  const T* Ty;
  const T* muA;   // [nlat]
  // preconditioner.  FP32 path: line-solve constants c, 1/w, z permuted
  // [nlat][C][32] (per-lane chunks).  FP64 path: the LU factors l, 1/w, u in
  // natural layout [nlat][nlon] and z natural.  Jacobi: the diagonal, natural.
  const T* lc;
  const T* lw;
  const T* lz;
  const T* lu;    // FP64 path: u_i = -Tx_i / w_i
  const T* lrow;  // [nlat][4]: FP32 path 1/delta, Tx_{n-1}/delta, Tx_{n-2}/delta; FP64 path delta and
                  // then the same three constants
  // FP64 path, lchunk = 1: the factors again in the per-lane chunk layout of
  // the FP32 path (c = -u, 1/w, z), for the chunked warp solve of a row
  // (rows of at least kChunkMinLon columns); lchunk = 0: the serial solve
  const T* lcc;
  const T* lwc;
  const T* lzc;
  int lchunk;
  // FP32 path, streamed solves: c = -u, 1/w, z in the piece-major layout of
  // the streamed rounds ([nlat][32][C + 4], zero past the leading block)
  const T* lcp;
  const T* lwp;
  const T* lzp;
  // Krylov vectors (inner precision)
  T* phi[3];
  T* r[3];
  T* e[2];   // e = P^-1 r and L(e), double-buffered in the mixed path (a fused
  T* Le[2];  // step reads the previous step's while writing its own)
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
  double* part;      // [2][nt][kNPart][2] double-double partial sums
  SolveState* st;    // [2]
  SolveState* result;  // final record (written once)
  const Fault* faults;
  double* patchval;  // [kMaxFaults]
  const LossEv* losses;  // [kMaxLosses]
  int nlosses;
  int protect;  // 0: plain GCR(k), no fault test (the paper's unprotected runs)
  // split rounds: the step phases run as two passes over the tiles with a
  // grid barrier between them (no recomputed halo rows); cs_off: offset of
  // the staged line-solve constants in the dynamic shared memory (elements);
  // cs_clobber: the second pass's rows overlap them
  // split 2: streamed step rounds (one tall band per CTA, rows streamed
  // through nslot shared-memory stage buffers); its other rounds run as
  // split rounds over sub-bands of at most sub_h rows (0: the whole tile)
  int split, cs_off, cs_clobber;
  int sub_h, nslot;
  // FP64 line solve: the factors are read from global memory, not staged
  // (wide rows, where staging them would leave bands thinner than the SM
  // count gives)
  int cs_global;
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

// Double-double pair (unnormalised hi + lo), the carrier of every partial sum.
struct DD {
  double hi, lo;
};
// Sum of two pairs: TwoSum of the leading parts, trailing parts added.
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  const double t = a.hi + b.hi;
  const double z = t - a.hi;
  const double q = (a.hi - (t - z)) + (b.hi - z);
  return DD{t, (a.lo + b.lo) + q};
}

// Inner-product accumulators.  FP64 vectors, with mode(1) (the solve's
// oracle order): Dot2 (Ogita, Rump and Oishi): exact products by fma
// (TwoProduct), running sum by TwoSum, low parts collected; the same
// algorithm as the CPU oracle's inner product, so both round (p + s) of
// nearly the same double-double value.  With mode(0), the default: one fma
// per element within the thread, double-double from the warp up; the sum then
// differs from Dot2's by about the rounding of a few hundred terms (relative
// 1e-14 at most), far below the margins of the fault test.  FP32 vectors: the
// product of two floats is exact as a float pair (TwoProduct with fmaf) and is
// accumulated in a float-float pair; warps combine float-float pairs in FP32
// and only per-warp sums reach FP64 (GB300's FP64 pipe is ~60x slower than
// FP32).
template <typename T>
struct Acc;
template <>
struct Acc<double> {
  double p, s;
  bool ex;  // Dot2 within the thread, else one fma per element
  __device__ __forceinline__ Acc() : p(0.0), s(0.0), ex(true) {}
  __device__ __forceinline__ void mode(int dot2) { ex = dot2 != 0; }
  __device__ __forceinline__ void add(double a, double b) {
    if (!ex) {
      // each thread's few hundred products by fma; the sums above the thread
      // stay double-double.  GB300 issues about two FP64 operations per SM
      // and clock, so the eight of TwoProduct + TwoSum per element cost more
      // than the rest of a step together.
      p = fma(a, b, p);
      return;
    }
    const double h = a * b;
    const double r = fma(a, b, -h);
    const double t = p + h;
    const double z = t - p;
    const double q = (p - (t - z)) + (h - z);
    p = t;
    s = s + (q + r);
  }
  // sum over the warp (xor butterfly, identical order in every warp)
  __device__ __forceinline__ DD warp_sum() const {
    DD v{p, s};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      DD w{__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o)};
      v = dd_add(v, w);
    }
    return v;
  }
};
// Plain FP64 accumulation (one fma per element), for the mixed path's outer
// residual norm: its decisions need FP64 accuracy, not the oracle's
// compensated sum, and GB300's FP64 pipe makes each extra operation costly.
struct AccF64 {
  double s;
  __device__ __forceinline__ AccF64() : s(0.0) {}
  __device__ __forceinline__ void add(double a, double b) { s = fma(a, b, s); }
  __device__ __forceinline__ DD warp_sum() const {
    double v = s;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return DD{v, 0.0};
  }
};
template <>
struct Acc<float> {
  float hi, lo;
  __device__ __forceinline__ Acc() : hi(0.f), lo(0.f) {}
  __device__ __forceinline__ void mode(int) {}  // always compensated (FP32 pipe)
  __device__ __forceinline__ void add(float a, float b) {
    const float p = a * b;
    const float pe = fmaf(a, b, -p);
    const float s = hi + p;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (p - bb);
    hi = s;
    lo = lo + (err + pe);
  }
  __device__ __forceinline__ DD warp_sum() const {
    float h = hi, l = lo;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const float h2 = __shfl_xor_sync(0xffffffffu, h, o);
      const float l2 = __shfl_xor_sync(0xffffffffu, l, o);
      const float t = h + h2;
      const float z = t - h;
      const float q = (h - (t - z)) + (h2 - z);
      h = t;
      l = (l + l2) + q;
    }
    return DD{(double)h, (double)l};
  }
};

// Per-CTA partial sums: each warp contributes its DD sum of every value; the
// CTA combines the warps' pairs in a fixed binary tree (depth 3 for 8 warps:
// GB300's FP64 latency makes a serial chain expensive) and writes nv pairs.
// FP64 path: double-double adds; FP32 path: each warp pair is first rounded to
// one double, then plain FP64 adds.
struct CtaRed {
  DD w[kWarps][kNPart];
};
__device__ __forceinline__ void cta_red_put(CtaRed& cr, int v, DD x) {
  if ((threadIdx.x & 31) == 0) cr.w[threadIdx.x >> 5][v] = x;
}
template <typename T>
__device__ __forceinline__ void cta_red_finish(CtaRed& cr, int nv, double* out, int v0 = 0) {
  __syncthreads();
  if (threadIdx.x >= v0 && threadIdx.x < nv) {
    const int v = threadIdx.x;
    if constexpr (sizeof(T) == 8) {
      DD t[kWarps];
#pragma unroll
      for (int w = 0; w < kWarps; ++w) t[w] = cr.w[w][v];
#pragma unroll
      for (int h = 1; h < kWarps; h <<= 1)
#pragma unroll
        for (int w = 0; w + h < kWarps; w += 2 * h) t[w] = dd_add(t[w], t[w + h]);
      out[2 * v] = t[0].hi;
      out[2 * v + 1] = t[0].lo;
    } else {
      double t[kWarps];
#pragma unroll
      for (int w = 0; w < kWarps; ++w) t[w] = cr.w[w][v].hi + cr.w[w][v].lo;
#pragma unroll
      for (int h = 1; h < kWarps; h <<= 1)
#pragma unroll
        for (int w = 0; w + h < kWarps; w += 2 * h) t[w] = t[w] + t[w + h];
      out[2 * v] = t[0];
      out[2 * v + 1] = 0.0;
    }
  }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// 16-byte vector access (4 floats or 2 doubles), L2-coherent loads.
template <typename T>
struct V16 {
  static constexpr int W = 16 / sizeof(T);
  T v[W];
};
template <typename T>
__device__ __forceinline__ V16<T> ldv(const T* p) {
  const uint4 u = __ldcg(reinterpret_cast<const uint4*>(p));
  V16<T> r;
  memcpy(&r, &u, 16);
  return r;
}
template <typename T>
__device__ __forceinline__ V16<T> ldv_nc(const T* p) {
  const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
  V16<T> r;
  memcpy(&r, &u, 16);
  return r;
}
template <typename T>
__device__ __forceinline__ void stv(T* p, const V16<T>& x) {
  uint4 u;
  memcpy(&u, &x, 16);
  *reinterpret_cast<uint4*>(p) = u;
}

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_s(unsigned smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

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
    // arrive with release semantics (the block's writes, ordered before by the
    // block barrier, become visible with the count), wait with acquire loads
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(counter), "r"(1u) : "memory");
    unsigned long long t0 = globaltimer();
    unsigned int it = 0;
    while (ld_acquire_u32(counter) < target) {
      if ((++it & 63u) == 0u && globaltimer() - t0 > kBarrierTimeoutNs) {
        atomicExch(err, 1);
        break;
      }
      __nanosleep(20);
    }
    *bail_smem = ld_acquire_u32(reinterpret_cast<const unsigned int*>(err));
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

// The same operator with fused multiply-adds (9 FP64 operations instead of
// 13): the mixed path's FP64 refinement residual, whose value needs FP64
// accuracy but not the oracle's operation order.
__device__ __forceinline__ double stencil5_fma(double v, double ve, double vw, double vn, double vs, double txc,
                                               double txw, double tyc, double tys, double muA, bool hasN, bool hasS) {
  double s = -muA * v;
  if (hasS) s = fma(tys, vs - v, s);
  if (hasN) s = fma(tyc, vn - v, s);
  s = fma(txw, vw - v, s);
  return fma(txc, ve - v, s);
}

// The solve's operator: FP32 vectors in the oracle's form; FP64 vectors in it
// only in the oracle's operation order, else with fused multiply-adds.
template <typename T>
__device__ __forceinline__ T stencil_op(int oracle_order, T v, T ve, T vw, T vn, T vs, T txc, T txw, T tyc, T tys,
                                        T muA, bool hasN, bool hasS) {
  if constexpr (sizeof(T) == 8) {
    if (!oracle_order) return stencil5_fma(v, ve, vw, vn, vs, txc, txw, tyc, tys, muA, hasN, hasS);
  }
  return stencil5<T>(v, ve, vw, vn, vs, txc, txw, tyc, tys, muA, hasN, hasS);
}

// Shared-memory row layout: element i of a row lives at i + i/32 (one pad
// word per 32), which keeps both the coalesced sweeps and the per-lane
// contiguous chunks of the line solve free of bank conflicts.
__host__ __device__ __forceinline__ int sk(int i) { return i + (i >> 5); }

// Elements per lane of the FP32 line solve: the n-1 unknowns of the row's
// leading block over 32 lanes, rounded up to whole register blocks of 8 (the
// solve runs every lane's chunk in full; positions past the block carry zero
// factors).
__host__ __device__ __forceinline__ int chunk_len(int nlon) {
  const int c = (nlon - 1 + 31) / 32;
  return (c + 7) & ~7;
}

// Floats (or doubles) per staged row: the row, its pad words, and room for the
// line solve's padded chunk positions.
__host__ __device__ __forceinline__ int row_stride(int nlon) {
  const int pad = 32 * chunk_len(nlon) + 1;
  const int ne = nlon > pad ? nlon : pad;
  int s = ne + (ne >> 5) + 1;
  return (s + 3) & ~3;
}

// ----------------------------------------------------------- line solve
// Row-local line-solve constants in the per-lane chunk layout [k][lane]
// (element i = lane*C + k): c_i = Tx_i / w_i, winv_i = 1 / w_i, z_i.  The
// pointers may address shared memory (staged by the caller) or global memory.
// Explicit shared-memory accesses.  An out-of-line device function receives
// shared-memory pointers as generic pointers and, not knowing their state
// space, accesses them through the slower generic path; the row solves below
// take the 32-bit shared address once and use ld.shared / st.shared.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
template <typename T>
__device__ __forceinline__ T lds(unsigned a);
template <>
__device__ __forceinline__ float lds<float>(unsigned a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a));
  return v;
}
template <>
__device__ __forceinline__ double lds<double>(unsigned a) {
  double v;
  asm volatile("ld.shared.f64 %0, [%1];" : "=d"(v) : "r"(a));
  return v;
}
__device__ __forceinline__ void sts(unsigned a, float v) { asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory"); }
__device__ __forceinline__ void sts(unsigned a, double v) { asm volatile("st.shared.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory"); }

template <typename T>
struct LineConsts {
  const T* cb;
  const T* cw;
  const T* cz;
};

template <typename T>
__device__ __forceinline__ LineConsts<T> line_consts_global(const SolveDev<T>& sd, int j) {
  const long long o = (long long)j * 32 * sd.C;
  return LineConsts<T>{sd.lc + o, sd.lw + o, sd.lz + o};
}

constexpr int kLB = 8;
constexpr int kChunkMinLon = 256;  // FP64 path: the chunked row solve from this row width  // register block of the recurrences

// Periodic tridiagonal solve of one latitude row, M e = -r (P = -M is the
// zonal part of L plus the diagonal of the rest), in place in shared memory,
// by one warp.  The leading (n-1) x (n-1) block uses its precomputed LU
// factorisation: forward g_i = b_i + c_{i-1} g_{i-1} (b = -r), backward
// y_i = winv_i g_i + c_i y_{i+1}.  Each recurrence runs over 32 contiguous
// per-lane chunks: a read-only pass forms each chunk's affine map, a warp
// scan composes the maps into each chunk's carry-in, and a second pass
// replays the chunk from its exact carry-in.  The periodic coupling of the
// last unknown is eliminated by bordering with the precomputed
// z = A0^-1 (-Tx_{n-1} e_0 - Tx_{n-2} e_{n-2}).  row must be in shared
// memory; the constants too, or (GC) in global memory in the same layout.
template <typename T, bool GC = false>
__device__ __noinline__ void line_solve_row(const SolveDev<T>& sd, int j, T* row_, const LineConsts<T> lc) {
  const int lane = threadIdx.x & 31;
  const int n = sd.nlon, m = n - 1, C = sd.C;
  const int i0 = lane * C;
  const int len = C;  // every lane runs its whole chunk (chunk_len)
  // the row's bordering constants, loaded first so that their latency hides
  // behind the recurrences
  // (FP64 path: after delta in slot 0)
  const T* lr = sd.lrow + (long long)j * 4 + (sizeof(T) == 8 ? 1 : 0);
  const T lr0 = __ldg(lr + 0), lr1 = __ldg(lr + 1), lr2 = __ldg(lr + 2);
  const unsigned rb = smem_addr(row_), cbb = smem_addr(lc.cb), cwb = smem_addr(lc.cw), czb = smem_addr(lc.cz);
  constexpr unsigned E = sizeof(T);
  auto R = [&](int i) { return rb + E * (unsigned)sk(i); };
  auto Cb = [&](int k) { return cbb + E * (unsigned)(k * 32 + lane); };
  auto Cw = [&](int k) { return cwb + E * (unsigned)(k * 32 + lane); };
  auto Cz = [&](int k) { return czb + E * (unsigned)(k * 32 + lane); };
  // the constants: shared memory, or (GC) global memory in the same layout
  auto cB = [&](int k) { return GC ? __ldg(lc.cb + k * 32 + lane) : lds<T>(Cb(k)); };
  auto cW = [&](int k) { return GC ? __ldg(lc.cw + k * 32 + lane) : lds<T>(Cw(k)); };
  auto cZ = [&](int k) { return GC ? __ldg(lc.cz + k * 32 + lane) : lds<T>(Cz(k)); };
  // b_{n-1}, read before the passes: its slot may lie in the last lane's chunk
  const T bl = -lds<T>(R(n - 1));
  // positions past the row hold no data: make them finite (their factors are zero)
  if (i0 + C > n)
    for (int k = 0; k < C; ++k)
      if (i0 + k >= n) sts(R(i0 + k), T(0));
  __syncwarp();
  // forward multiplier of chunk element 0 is c_{i0-1}, the last c of the previous lane
  const T mylast = cB(C - 1);
  T a0 = __shfl_up_sync(0xffffffffu, mylast, 1);
  if (lane == 0) a0 = T(0);
  // pass 1: affine map g_out = F g_in + G of the chunk
  T F = T(1), G = T(0);
  {
    T a = a0;
    for (int kb = 0; kb < len; kb += kLB) {
      T rv[kLB], cv[kLB];
#pragma unroll
      for (int q = 0; q < kLB; ++q) {
        rv[q] = lds<T>(R(i0 + kb + q));
        cv[q] = cB(kb + q);
      }
#pragma unroll
      for (int q = 0; q < kLB; ++q) {
        G = tfma(a, G, -rv[q]);
        F = F * a;
        a = cv[q];
      }
    }
  }
  T Fs = F, Gs = G;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T Fo = __shfl_up_sync(0xffffffffu, Fs, d);
    const T Go = __shfl_up_sync(0xffffffffu, Gs, d);
    if (lane >= d) {
      Gs = tfma(Fs, Go, Gs);
      Fs = Fs * Fo;
    }
  }
  T carry = __shfl_up_sync(0xffffffffu, Gs, 1);
  if (lane == 0) carry = T(0);
  // pass 2: g from the exact carry-in
  {
    T a = a0, g = carry;
    for (int kb = 0; kb < len; kb += kLB) {
      T rv[kLB], cv[kLB];
#pragma unroll
      for (int q = 0; q < kLB; ++q) {
        rv[q] = lds<T>(R(i0 + kb + q));
        cv[q] = cB(kb + q);
      }
#pragma unroll
      for (int q = 0; q < kLB; ++q) {
        g = tfma(a, g, -rv[q]);
        rv[q] = g;
        a = cv[q];
      }
#pragma unroll
      for (int q = 0; q < kLB; ++q)
        sts(R(i0 + kb + q), rv[q]);
    }
  }
  // pass 3: affine map of the backward recurrence y_in = Fb y_out + Y
  const int kb_last = len > 0 ? ((len - 1) / kLB) * kLB : -1;
  T Fb = T(1), Y = T(0);
  for (int kb = kb_last; kb >= 0; kb -= kLB) {
    T gv[kLB], cv[kLB], wv[kLB];
#pragma unroll
    for (int q = 0; q < kLB; ++q) {
      gv[q] = lds<T>(R(i0 + kb + q));
      cv[q] = cB(kb + q);
      wv[q] = cW(kb + q);
    }
#pragma unroll
    for (int q = kLB - 1; q >= 0; --q) {
      Y = tfma(cv[q], Y, gv[q] * wv[q]);
      Fb = Fb * cv[q];
    }
  }
  T Fr = Fb, Yr = Y;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const T Fo = __shfl_down_sync(0xffffffffu, Fr, d);
    const T Yo = __shfl_down_sync(0xffffffffu, Yr, d);
    if (lane + d < 32) {
      Yr = tfma(Fr, Yo, Yr);
      Fr = Fr * Fo;
    }
  }
  T carryb = __shfl_down_sync(0xffffffffu, Yr, 1);
  if (lane == 31) carryb = T(0);
  // pass 4: y from the exact carry-in
  {
    T y = carryb;
    for (int kb = kb_last; kb >= 0; kb -= kLB) {
      T gv[kLB], cv[kLB], wv[kLB];
#pragma unroll
      for (int q = 0; q < kLB; ++q) {
        gv[q] = lds<T>(R(i0 + kb + q));
        cv[q] = cB(kb + q);
        wv[q] = cW(kb + q);
      }
#pragma unroll
      for (int q = kLB - 1; q >= 0; --q) {
        y = tfma(cv[q], y, gv[q] * wv[q]);
        gv[q] = y;
      }
#pragma unroll
      for (int q = 0; q < kLB; ++q)
        sts(R(i0 + kb + q), gv[q]);
    }
  }
  __syncwarp();
  // bordering: x_{n-1} = (b_{n-1} + Tx_{n-1} y_0 + Tx_{n-2} y_{m-1}) / delta
  const T y0 = lds<T>(R(0));
  const T ym = lds<T>(R(m - 1));
  const T xl = tfma(lr2, ym, tfma(lr1, y0, bl * lr0));
  __syncwarp();
#pragma unroll 8
  for (int k = 0; k < len; ++k) sts(R(i0 + k), tfma(-xl, cZ(k), lds<T>(R(i0 + k))));
  __syncwarp();
  if (lane == 0) sts(R(n - 1), xl);
  __syncwarp();
}

// The same solve of one row by a group of G warps (G = 2, 4 or 8), for tiles
// with fewer rows than warps.  Thread (w, lane) of the group takes piece
// p = lane * G + w of the row: elements lane * C + w * C/G + kk, kk < C/G, so
// the pieces run in row order and the constants keep their per-lane layout.
// Each recurrence: every piece's affine map (pass 1 / 3) into `maps`, a group
// barrier, each lane composes the maps of its G pieces, a warp scan over the
// lanes gives every lane's carry-in, and each piece applies its lane's earlier
// pieces to it; then the piece is replayed from its exact carry-in (pass 2 /
// 4).  C must be a multiple of 8 G.  `maps`: 2 * 32 * G floats of shared
// memory per group; `bar`: the group's named barrier (1..15).
__device__ __forceinline__ void group_sync(int bar, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nthreads) : "memory");
}
template <int G>
__device__ __noinline__ void line_solve_row_group(const SolveDev<float>& sd, int j, float* row_,
                                                  const LineConsts<float> lc, float* maps, int bar) {
  const int lane = threadIdx.x & 31, w = (threadIdx.x >> 5) % G;
  const int n = sd.nlon, m = n - 1, C = sd.C, Cp = C / G;
  const int i0 = lane * C + w * Cp, k0 = w * Cp;
  const float* lr = sd.lrow + (long long)j * 4;
  const float lr0 = __ldg(lr + 0), lr1 = __ldg(lr + 1), lr2 = __ldg(lr + 2);
  const unsigned rb = smem_addr(row_), cbb = smem_addr(lc.cb), cwb = smem_addr(lc.cw), czb = smem_addr(lc.cz);
  auto R = [&](int i) { return rb + 4u * (unsigned)sk(i); };
  auto Cb = [&](int k) { return cbb + 4u * (unsigned)(k * 32 + lane); };
  auto Cw = [&](int k) { return cwb + 4u * (unsigned)(k * 32 + lane); };
  auto Cz = [&](int k) { return czb + 4u * (unsigned)(k * 32 + lane); };
  float* mF = maps;           // [G][32]
  float* mG = maps + 32 * G;  // [G][32]
  const float bl = -lds<float>(R(n - 1));
  if (i0 + Cp > n)
    for (int kk = 0; kk < Cp; ++kk)
      if (i0 + kk >= n) sts(R(i0 + kk), 0.f);
  // forward multiplier of the piece's first element: c of the element before
  float a0 = 0.f;
  if (w > 0)
    a0 = lds<float>(Cb(k0 - 1));
  else if (lane > 0)
    a0 = lds<float>(cbb + 4u * (unsigned)((C - 1) * 32 + lane - 1));
  // pass 1: the piece's map g_out = F g_in + Gm
  float F = 1.f, Gm = 0.f;
  {
    float a = a0;
    for (int kb = 0; kb < Cp; kb += kLB) {
      float rv[kLB], cv[kLB];
#pragma unroll
      for (int q = 0; q < kLB; ++q) {
        rv[q] = lds<float>(R(i0 + kb + q));
        cv[q] = lds<float>(Cb(k0 + kb + q));
      }
#pragma unroll
      for (int q = 0; q < kLB; ++q) {
        Gm = tfma(a, Gm, -rv[q]);
        F = F * a;
        a = cv[q];
      }
    }
  }
  mF[w * 32 + lane] = F;
  mG[w * 32 + lane] = Gm;
  group_sync(bar, 32 * G);
  float FL = 1.f, GL = 0.f, Fw[G], Gw[G];
#pragma unroll
  for (int q = 0; q < G; ++q) {
    Fw[q] = mF[q * 32 + lane];
    Gw[q] = mG[q * 32 + lane];
    GL = tfma(Fw[q], GL, Gw[q]);
    FL = FL * Fw[q];
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Fo = __shfl_up_sync(0xffffffffu, FL, d);
    const float Go = __shfl_up_sync(0xffffffffu, GL, d);
    if (lane >= d) {
      GL = tfma(FL, Go, GL);
      FL = FL * Fo;
    }
  }
  float carry = __shfl_up_sync(0xffffffffu, GL, 1);
  if (lane == 0) carry = 0.f;
#pragma unroll
  for (int q = 0; q < G; ++q)
    if (q < w) carry = tfma(Fw[q], carry, Gw[q]);
  // pass 2: g from the exact carry-in
  {
    float a = a0, g = carry;
    for (int kb = 0; kb < Cp; kb += kLB) {
      float rv[kLB], cv[kLB];
#pragma unroll
      for (int q = 0; q < kLB; ++q) {
        rv[q] = lds<float>(R(i0 + kb + q));
        cv[q] = lds<float>(Cb(k0 + kb + q));
      }
#pragma unroll
      for (int q = 0; q < kLB; ++q) {
        g = tfma(a, g, -rv[q]);
        rv[q] = g;
        a = cv[q];
      }
#pragma unroll
      for (int q = 0; q < kLB; ++q) sts(R(i0 + kb + q), rv[q]);
    }
  }
  group_sync(bar, 32 * G);  // every carry read before the maps are reused
  // pass 3: the piece's backward map y_in = Fb y_out + Y
  float Fb = 1.f, Y = 0.f;
  for (int kb = Cp - kLB; kb >= 0; kb -= kLB) {
    float gv[kLB], cv[kLB], wv[kLB];
#pragma unroll
    for (int q = 0; q < kLB; ++q) {
      gv[q] = lds<float>(R(i0 + kb + q));
      cv[q] = lds<float>(Cb(k0 + kb + q));
      wv[q] = lds<float>(Cw(k0 + kb + q));
    }
#pragma unroll
    for (int q = kLB - 1; q >= 0; --q) {
      Y = tfma(cv[q], Y, gv[q] * wv[q]);
      Fb = Fb * cv[q];
    }
  }
  mF[w * 32 + lane] = Fb;
  mG[w * 32 + lane] = Y;
  group_sync(bar, 32 * G);
  float FbL = 1.f, YL = 0.f;
#pragma unroll
  for (int q = G - 1; q >= 0; --q) {
    Fw[q] = mF[q * 32 + lane];
    Gw[q] = mG[q * 32 + lane];
    YL = tfma(Fw[q], YL, Gw[q]);
    FbL = FbL * Fw[q];
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Fo = __shfl_down_sync(0xffffffffu, FbL, d);
    const float Yo = __shfl_down_sync(0xffffffffu, YL, d);
    if (lane + d < 32) {
      YL = tfma(FbL, Yo, YL);
      FbL = FbL * Fo;
    }
  }
  float carryb = __shfl_down_sync(0xffffffffu, YL, 1);
  if (lane == 31) carryb = 0.f;
#pragma unroll
  for (int q = G - 1; q >= 0; --q)
    if (q > w) carryb = tfma(Fw[q], carryb, Gw[q]);
  // pass 4: y from the exact carry-in
  {
    float y = carryb;
    for (int kb = Cp - kLB; kb >= 0; kb -= kLB) {
      float gv[kLB], cv[kLB], wv[kLB];
#pragma unroll
      for (int q = 0; q < kLB; ++q) {
        gv[q] = lds<float>(R(i0 + kb + q));
        cv[q] = lds<float>(Cb(k0 + kb + q));
        wv[q] = lds<float>(Cw(k0 + kb + q));
      }
#pragma unroll
      for (int q = kLB - 1; q >= 0; --q) {
        y = tfma(cv[q], y, gv[q] * wv[q]);
        gv[q] = y;
      }
#pragma unroll
      for (int q = 0; q < kLB; ++q) sts(R(i0 + kb + q), gv[q]);
    }
  }
  group_sync(bar, 32 * G);
  // bordering: x_{n-1} = (b_{n-1} + Tx_{n-1} y_0 + Tx_{n-2} y_{m-1}) / delta
  const float y0 = lds<float>(R(0));
  const float ym = lds<float>(R(m - 1));
  const float xl = tfma(lr2, ym, tfma(lr1, y0, bl * lr0));
  group_sync(bar, 32 * G);
#pragma unroll 8
  for (int kk = 0; kk < Cp; ++kk) sts(R(i0 + kk), tfma(-xl, lds<float>(Cz(k0 + kk)), lds<float>(R(i0 + kk))));
  group_sync(bar, 32 * G);
  if (lane == 0 && w == 0) sts(R(n - 1), xl);
}

// FP64 path: the row's periodic tridiagonal solve by ONE thread, operation for
// operation the CPU oracle's Thomas substitution: forward y_0 = b_0,
// y_i = fma(-l_i, y_{i-1}, b_i); backward y_{m-1} = y_{m-1} winv_{m-1},
// y_i = fma(-u_i, y_{i+1}, y_i winv_i); bordering x_{n-1} = (b_{n-1} +
// Tx_{n-1} y_0 + Tx_{n-2} y_{m-1}) / delta, x_i = y_i - x_{n-1} z_i; b = -r.
// Bitwise reproducible against the oracle.  l, winv, u: the row's factors in
// natural layout (shared or global memory).
static __device__ __noinline__ void line_solve_row_seq(const SolveDev<double>& sd, int j, double* row, const double* l,
                                   const double* winv, const double* u) {
  const int n = sd.nlon, m = n - 1;
  double y = -row[sk(0)];
  row[sk(0)] = y;
  for (int i0 = 1; i0 < m; i0 += kLB) {
    double bv[kLB], lv[kLB];
#pragma unroll
    for (int q = 0; q < kLB; ++q)
      if (i0 + q < m) {
        bv[q] = -row[sk(i0 + q)];
        lv[q] = l[i0 + q];
      }
#pragma unroll
    for (int q = 0; q < kLB; ++q)
      if (i0 + q < m) {
        y = fma(-lv[q], y, bv[q]);
        bv[q] = y;
      }
#pragma unroll
    for (int q = 0; q < kLB; ++q)
      if (i0 + q < m) row[sk(i0 + q)] = bv[q];
  }
  y = row[sk(m - 1)] * winv[m - 1];
  row[sk(m - 1)] = y;
  for (int i1 = m - 2; i1 >= 0; i1 -= kLB) {  // block [i1 - kLB + 1, i1], descending
    double gv[kLB], wv[kLB], uv[kLB];
#pragma unroll
    for (int q = 0; q < kLB; ++q)
      if (i1 - q >= 0) {
        gv[q] = row[sk(i1 - q)];
        wv[q] = winv[i1 - q];
        uv[q] = u[i1 - q];
      }
#pragma unroll
    for (int q = 0; q < kLB; ++q)
      if (i1 - q >= 0) {
        y = fma(-uv[q], y, gv[q] * wv[q]);
        gv[q] = y;
      }
#pragma unroll
    for (int q = 0; q < kLB; ++q)
      if (i1 - q >= 0) row[sk(i1 - q)] = gv[q];
  }
  const double* tx = sd.Tx + (long long)j * n;
  const double* z = sd.lz + (long long)j * n;
  const double num = -row[sk(n - 1)] + __ldg(tx + n - 1) * row[sk(0)] + __ldg(tx + n - 2) * row[sk(m - 1)];
  const double xl = num / __ldg(sd.lrow + (long long)j * 4);
#pragma unroll 8
  for (int i = 0; i < m; ++i) row[sk(i)] = row[sk(i)] - xl * __ldg(z + i);
  row[sk(n - 1)] = xl;
}

// Pointwise preconditioners on a shared-memory row (one warp).  Jacobi:
// e = -r / d (FP64 path: division, as the oracle) or -r (1/d) (FP32 path).
template <typename T>
__device__ void pointwise_precond_row(const SolveDev<T>& sd, int j, T* row) {
  const int lane = threadIdx.x & 31;
  if (sd.precond == PC_JACOBI) {
    const T* dg = sd.lw + (long long)j * sd.nlon;
    for (int i = lane; i < sd.nlon; i += 32) {
      if constexpr (sizeof(T) == 8)
        row[sk(i)] = -row[sk(i)] / __ldg(dg + i);
      else
        row[sk(i)] = -row[sk(i)] * __ldg(dg + i);
    }
  }
  __syncwarp();
}

// The same serial solve with the row and its factors in shared memory
// (explicit ld.shared / st.shared), split in three so that only the two
// dependent chains run lane-serial.  The backward step's product g_i winv_i
// does not depend on the chain: the caller forms it for all rows block-wide
// between the passes (the same rounded product, so the same values), and
// applies x_i = y_i - x_{n-1} z_i block-wide after them.  GB300's FP64 unit
// takes 64 cycles per warp instruction whatever the active lanes, so each
// FP64 instruction moved off a chain saves 64 cycles per element.  Whole
// blocks of kLB elements carry no per-element bounds tests (a scalar loop
// takes the remainder), which lets the block's loads issue together.
// Forward pass: y_0 = b_0, y_i = fma(-l_i, y_{i-1}, b_i), b = -r, i < m.
static __device__ __noinline__ void line_solve_fwd_sh(int n, double* row_, const double* l_) {
  const int m = n - 1;
  const unsigned rb = smem_addr(row_), lb = smem_addr(l_);
  auto R = [&](int i) { return rb + 8u * (unsigned)sk(i); };
  auto Lf = [&](int i) { return lb + 8u * (unsigned)i; };
  double y = -lds<double>(R(0));
  sts(R(0), y);
  int i0 = 1;
  for (; i0 + kLB <= m; i0 += kLB) {
    double bv[kLB], lv[kLB];
#pragma unroll
    for (int q = 0; q < kLB; ++q) {
      bv[q] = -lds<double>(R(i0 + q));
      lv[q] = lds<double>(Lf(i0 + q));
    }
#pragma unroll
    for (int q = 0; q < kLB; ++q) {
      y = fma(-lv[q], y, bv[q]);
      bv[q] = y;
    }
#pragma unroll
    for (int q = 0; q < kLB; ++q) sts(R(i0 + q), bv[q]);
  }
  for (; i0 < m; ++i0) {
    y = fma(-lds<double>(Lf(i0)), y, -lds<double>(R(i0)));
    sts(R(i0), y);
  }
}
// Backward pass on the products gw_i = g_i winv_i (i < m) already in the row:
// y_{m-1} = gw_{m-1}, y_i = fma(-u_i, y_{i+1}, gw_i); then
// x_{n-1} = (b_{n-1} + Tx_{n-1} y_0 + Tx_{n-2} y_{m-1}) / delta into slot n-1.
static __device__ __noinline__ void line_solve_bwd_sh(const SolveDev<double>& sd, int j, double* row_, const double* u_) {
  const int n = sd.nlon, m = n - 1;
  const unsigned rb = smem_addr(row_), ub = smem_addr(u_);
  auto R = [&](int i) { return rb + 8u * (unsigned)sk(i); };
  auto Uf = [&](int i) { return ub + 8u * (unsigned)i; };
  double y = lds<double>(R(m - 1));
  int i1 = m - 2;
  for (; i1 - kLB + 1 >= 0; i1 -= kLB) {  // block [i1 - kLB + 1, i1], descending
    double gv[kLB], uv[kLB];
#pragma unroll
    for (int q = 0; q < kLB; ++q) {
      gv[q] = lds<double>(R(i1 - q));
      uv[q] = lds<double>(Uf(i1 - q));
    }
#pragma unroll
    for (int q = 0; q < kLB; ++q) {
      y = fma(-uv[q], y, gv[q]);
      gv[q] = y;
    }
#pragma unroll
    for (int q = 0; q < kLB; ++q) sts(R(i1 - q), gv[q]);
  }
  for (; i1 >= 0; --i1) {
    y = fma(-lds<double>(Uf(i1)), y, lds<double>(R(i1)));
    sts(R(i1), y);
  }
  const double* tx = sd.Tx + (long long)j * n;
  const double num = -lds<double>(R(n - 1)) + __ldg(tx + n - 1) * lds<double>(R(0)) + __ldg(tx + n - 2) * lds<double>(R(m - 1));
  sts(R(n - 1), num / __ldg(sd.lrow + (long long)j * 4));
}

// The two chains with the factors l and u kept in global memory (FP64 path,
// wide rows): the same operations on the same values as line_solve_fwd_sh
// and line_solve_bwd_sh.  Each chain's lane copies its row's factors into a
// ring of kRingSlots chunks of kRingChunk elements in shared memory (ring_,
// its own, 16-byte aligned), one chunk ahead of the chain, with cp.async
// (16-byte copies where the row starts on a 16-byte boundary, else 8-byte
// ones), and reads them from there: no global-memory latency and no prefetch
// registers on the chain.  Element i sits at ring position i mod kRingElems
// (chunk i / kRingChunk); a slot is reused once the chain has moved
// kRingSlots - 1 chunks on.
constexpr int kRingChunk = 64, kRingSlots = 4;
constexpr int kRingElems = kRingChunk * kRingSlots;  // a power of two
// rings of successive rows kRingStride doubles apart: 16 bytes more than a
// ring, so the rows side by side in lanes read different banks
constexpr int kRingStride = kRingElems + 2;
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void cp_async8(unsigned smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
// Chunk c of a row's factors f (elements [c kRingChunk, ...) below lim, lim <=
// n) into the ring at gb; always one commit group (empty for c < 0).  A
// 16-byte copy may take the element at lim too (still inside the row).
__device__ __forceinline__ void ring_fetch(unsigned gb, const double* f, int c, int lim, bool a16) {
  if (c >= 0) {
    const int i0 = c * kRingChunk, i1 = min(i0 + kRingChunk, lim);
    if (a16) {
      for (int i = i0; i < i1; i += 2) cp_async16_s(gb + 8u * (unsigned)(i & (kRingElems - 1)), f + i);
    } else {
      for (int i = i0; i < i1; ++i) cp_async8(gb + 8u * (unsigned)(i & (kRingElems - 1)), f + i);
    }
  }
  cp_async_commit();
}

static __device__ __noinline__ void line_solve_fwd_gl(int n, double* row_, const double* __restrict__ l, double* ring_) {
  const int m = n - 1;
  const unsigned rb = smem_addr(row_), gb = smem_addr(ring_);
  const bool a16 = (reinterpret_cast<unsigned long long>(l) & 15ull) == 0;
  auto R = [&](int i) { return rb + 8u * (unsigned)sk(i); };
  auto G = [&](int i) { return gb + 8u * (unsigned)(i & (kRingElems - 1)); };
  ring_fetch(gb, l, 0, m, a16);
  ring_fetch(gb, l, 1, m, a16);
  cp_async_wait_1();
  int ready = 0;  // chunks 0..ready have landed, ready + 1 is in flight
  double y = -lds<double>(R(0));
  sts(R(0), y);
  const int nb = (m - 1) / kLB;  // whole blocks from i = 1
  for (int b = 0; b < nb; ++b) {
    const int i0 = 1 + b * kLB;
    if ((i0 + kLB - 1) / kRingChunk > ready) {  // the block reaches the next chunk
      ++ready;
      ring_fetch(gb, l, ready + 1, m, a16);
      cp_async_wait_1();
    }
    double bv[kLB], lv[kLB];
#pragma unroll
    for (int q = 0; q < kLB; ++q) {
      bv[q] = -lds<double>(R(i0 + q));
      lv[q] = lds<double>(G(i0 + q));
    }
#pragma unroll
    for (int q = 0; q < kLB; ++q) {
      y = fma(-lv[q], y, bv[q]);
      bv[q] = y;
    }
#pragma unroll
    for (int q = 0; q < kLB; ++q) sts(R(i0 + q), bv[q]);
  }
  cp_async_wait_all();
  for (int i0 = 1 + nb * kLB; i0 < m; ++i0) {  // fewer than kLB: their factors straight from global memory
    y = fma(-__ldg(l + i0), y, -lds<double>(R(i0)));
    sts(R(i0), y);
  }
}
static __device__ __noinline__ void line_solve_bwd_gl(const SolveDev<double>& sd, int j, double* row_,
                                                      const double* __restrict__ u, double* ring_) {
  const int n = sd.nlon, m = n - 1;
  const unsigned rb = smem_addr(row_), gb = smem_addr(ring_);
  const bool a16 = (reinterpret_cast<unsigned long long>(u) & 15ull) == 0;
  auto R = [&](int i) { return rb + 8u * (unsigned)sk(i); };
  auto G = [&](int i) { return gb + 8u * (unsigned)(i & (kRingElems - 1)); };
  const int ctop = (m - 2) / kRingChunk;  // the chain runs i = m-2 .. 0, chunks ctop .. 0
  ring_fetch(gb, u, ctop, m - 1, a16);
  ring_fetch(gb, u, ctop - 1, m - 1, a16);
  cp_async_wait_1();
  int ready = ctop;  // chunks ctop..ready have landed, ready - 1 is in flight
  double y = lds<double>(R(m - 1));
  const int nb = (m - 1) / kLB;  // whole blocks descending from i = m - 2
  for (int b = 0; b < nb; ++b) {
    const int i1 = m - 2 - b * kLB;  // block [i1 - kLB + 1, i1], descending
    if ((i1 - kLB + 1) / kRingChunk < ready) {
      --ready;
      ring_fetch(gb, u, ready - 1, m - 1, a16);
      cp_async_wait_1();
    }
    double gv[kLB], uv[kLB];
#pragma unroll
    for (int q = 0; q < kLB; ++q) {
      gv[q] = lds<double>(R(i1 - q));
      uv[q] = lds<double>(G(i1 - q));
    }
#pragma unroll
    for (int q = 0; q < kLB; ++q) {
      y = fma(-uv[q], y, gv[q]);
      gv[q] = y;
    }
#pragma unroll
    for (int q = 0; q < kLB; ++q) sts(R(i1 - q), gv[q]);
  }
  cp_async_wait_all();
  for (int i1 = m - 2 - nb * kLB; i1 >= 0; --i1) {
    y = fma(-__ldg(u + i1), y, lds<double>(R(i1)));
    sts(R(i1), y);
  }
  const double* tx = sd.Tx + (long long)j * n;
  const double num = -lds<double>(R(n - 1)) + __ldg(tx + n - 1) * lds<double>(R(0)) + __ldg(tx + n - 2) * lds<double>(R(m - 1));
  sts(R(n - 1), num / __ldg(sd.lrow + (long long)j * 4));
}

// Preconditioner solve of one row by one warp.  FP32: the chunked warp
// solve; FP64: lane 0 runs the oracle-identical sequential solve.
template <typename T>
__device__ __forceinline__ void precond_row(const SolveDev<T>& sd, int j, T* row, const LineConsts<T> lc) {
  if (sd.precond == PC_LINE) {
    if constexpr (sizeof(T) == 8) {
      if ((threadIdx.x & 31) == 0) line_solve_row_seq(sd, j, row, lc.cb, lc.cw, lc.cz);
      __syncwarp();
    } else {
      line_solve_row(sd, j, row, lc);
    }
  } else {
    pointwise_precond_row(sd, j, row);
  }
}

// Global-memory line-solve constants of row j (FP32: chunk layout c, 1/w, z;
// FP64: natural-layout factors l, 1/w, u).
template <typename T>
__device__ __forceinline__ LineConsts<T> row_consts_global(const SolveDev<T>& sd, int j) {
  if constexpr (sizeof(T) == 8) {
    const long long o = (long long)j * sd.nlon;
    return LineConsts<T>{sd.lc + o, sd.lw + o, sd.lu + o};
  } else {
    return line_consts_global(sd, j);
  }
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
