// Phases of the persistent FT-GCR(k) kernel and the per-solve state machine.
//
// One inner step of Algorithm 1 takes two rounds (one grid barrier each):
//   PA  phi' = phi + beta p^nu, r' = r + beta L(p^nu), ||r'||^2,
//       e = P^-1(r') (row solves, one halo row each side recomputed),
//       L(e) and <L(e), L(p^l)> for l = 0..nu           (one pass over HBM)
//   PB  exit test, fault test, backup or restore, alpha_l,
//       p^{nu+1} = e + sum alpha_l p^l, L(p^{nu+1}) likewise,
//       <r', L(p^{nu+1})>, <L(p^{nu+1}), L(p^{nu+1})>     (one pass over HBM)
// The exit and fault decisions of step t are taken at the start of the round
// that follows PA, from the reduced partial sums; the PA work of a step that
// exits or is rejected is simply discarded.
#pragma once
#include "ftgcr_device.cuh"

namespace ftgcr {

constexpr int kMaxBatch = 1024;

struct FlipEnt {
  long long g;
  int vec, bit, q;
};

template <typename T>
struct Ctx {
  int kind, nu, zero_guess, xsrc_user, finzero, patched, first;
  int rin_R;  // INIT: r0 = -R (zero initial guess; mixed: the first inner solve), ||R||^2 in FP64
  long long t;           // PA: executed step; INIT/PB/RESTORE: step whose x/r/p/Ap flips are applied
  long long patch_step;  // step of the flips whose clean values the backup carries
  T beta;
  T alpha[kMaxK];
  const T* phiC;
  T* phiW;
  const T* rC;
  T* rW;
  const T* pnu;
  const T* lpnu;
  const T* pp[kMaxK];
  const T* lp[kMaxK];
  const T* lo[kMaxK];  // PF: L(p^l) of the previous step's directions (lp: this step's)
  int nuo;             // PF: nu of the previous step
  T* eW;               // PA, PF: e and L(e) written
  T* LeW;
  const T* eR;         // PF, PB: e and L(e) of the previous step
  const T* LeR;
  T* pnew;
  T* lpnew;
  T* phiCw;  // PB: current phi (x flips)
  T* rCw;    // PB: current r (r flips, written back)
  const T* phiS;
  const T* rS;
  const T* pS;
  const T* lpS;
  T* phiT;
  T* rT;
  T* pT;
  T* lpT;
  const double* xsrc;
  double* xdst;
  const T* d;
  const T* finsrc;
};

struct LaunchCtl {
  unsigned int counter;
  int err;
  long long round0;
  long long round_end;
  int nonfinite;  // set by the check of staged host inputs: one held a NaN or an infinity
};

// Optional per-round trace: for every (round, CTA) the global timer at the
// round start, after the state transitions, after the phase work and after
// the grid barrier, plus the phase kind of the CTA's first item.
struct TraceEnt {
  unsigned long long t0, t1, t2, t3;
  unsigned long long s0, s1, s2;  // sub-phase marks of the first item (PA: axpy, line solve, stencil)
  int kind, items;
};

template <typename T>
struct BatchArgs {
  SolveDev<T>* const* solves;  // [n]
  const int* nt;               // [n] tiles per solve
  int* active;                 // [2][n]
  int n;
  LaunchCtl* ctl;
  int max_rounds;
  TraceEnt* trace;             // [trace_rounds][gridDim] or null
  int trace_rounds;
  int* diag;                   // [gridDim][4]: round, phase kind, checkpoint, items (failure report)
};

// ------------------------------------------------------------ flips
__device__ __forceinline__ bool fault_is_state_vec(int v) { return v == V_X || v == V_R || v == V_P || v == V_AP; }

// Build, in shared memory, the flips of step `step` on vectors in `vmask`
// whose element lies in [g0, g1).  Thread 0 only.
template <typename T>
__device__ int collect_flips(const SolveDev<T>& sd, long long step, unsigned vmask, long long g0, long long g1,
                             FlipEnt* out) {
  int n = 0;
  for (int q = 0; q < sd.nfaults; ++q) {
    const Fault f = sd.faults[q];
    if (f.step == step && ((vmask >> f.vec) & 1u) && f.index >= g0 && f.index < g1) {
      out[n].g = f.index;
      out[n].vec = f.vec;
      out[n].bit = f.bit;
      out[n].q = q;
      ++n;
    }
  }
  return n;
}

template <typename T>
__device__ __forceinline__ T apply_flips(T v, long long g, int vec, int nfl, const FlipEnt* fl) {
  for (int q = 0; q < nfl; ++q)
    if (fl[q].g == g && fl[q].vec == vec) v = flip_bits(v, fl[q].bit);
  return v;
}

// Clean value of the backup at element g of vector vec while it still
// carries the initialisation flips (see the INIT phase).
template <typename T>
__device__ __forceinline__ T apply_patches(T v, long long g, int vec, int npt, const FlipEnt* pt,
                                           const double* patchval) {
  for (int q = 0; q < npt; ++q)
    if (pt[q].g == g && pt[q].vec == vec) v = (T)__ldcg(patchval + pt[q].q);
  return v;
}

template <typename T>
__device__ __forceinline__ int count_faults(const SolveDev<T>& sd, long long step, unsigned vmask) {
  int c = 0;
  for (int q = 0; q < sd.nfaults; ++q)
    if (sd.faults[q].step == step && ((vmask >> sd.faults[q].vec) & 1u)) ++c;
  return c;
}

constexpr unsigned kStateVecs = (1u << V_X) | (1u << V_R) | (1u << V_P) | (1u << V_AP);

template <typename T>
__device__ __forceinline__ int count_losses(const SolveDev<T>& sd, long long step) {
  int c = 0;
  for (int q = 0; q < sd.nlosses; ++q) c += sd.losses[q].step == step;
  return c;
}

// ------------------------------------------------------------ reductions
// Deterministic sum over the nt tiles of the partials buffer of the first nv
// values.  Warp v sums value v: lanes take tiles lane, lane+32, ... (all loads
// issued first), add them in tile order, then a fixed xor tree.  FP64 path:
// double-double arithmetic throughout, rounded once; FP32 path: plain FP64
// (per-tile values are already accurate sums).  Every CTA that works on the
// solve gets bitwise the same numbers.
// Warps w0..kWarps-1 take part (warp w0 + i sums values i, i + (kWarps - w0),
// ...); the order within a value is the same whichever warp sums it.
template <typename T>
__device__ __forceinline__ void reduce_partials(const double* part, int nt, int nv, double* red, int w0 = 0) {
  constexpr int B = 8;  // tiles loaded per batch per lane, summed in a binary tree
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (warp < w0) return;
  for (int v = warp - w0; v < nv; v += kWarps - w0) {
    DD acc{0.0, 0.0};
    double acc1 = 0.0;
    for (int t0 = lane; t0 < nt; t0 += 32 * B) {
      DD tv[B];
#pragma unroll
      for (int q = 0; q < B; ++q) {
        const int tau = t0 + 32 * q;
        tv[q] = DD{0.0, 0.0};
        if (tau < nt) {
          tv[q].hi = __ldcg(part + (long long)tau * kPartStride + 2 * v);
          tv[q].lo = __ldcg(part + (long long)tau * kPartStride + 2 * v + 1);
        }
      }
      if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int h = 1; h < B; h <<= 1)
#pragma unroll
          for (int q = 0; q + h < B; q += 2 * h) tv[q] = dd_add(tv[q], tv[q + h]);
        acc = dd_add(acc, tv[0]);
      } else {
        double t[B];
#pragma unroll
        for (int q = 0; q < B; ++q) t[q] = tv[q].hi + tv[q].lo;
#pragma unroll
        for (int h = 1; h < B; h <<= 1)
#pragma unroll
          for (int q = 0; q + h < B; q += 2 * h) t[q] = t[q] + t[q + h];
        acc1 = acc1 + t[0];
      }
    }
    if constexpr (sizeof(T) == 8) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        acc = dd_add(acc, DD{__shfl_xor_sync(0xffffffffu, acc.hi, o), __shfl_xor_sync(0xffffffffu, acc.lo, o)});
      if (lane == 0) red[v] = acc.hi + acc.lo;
    } else {
      acc1 = warp_sum(acc1);
      if (lane == 0) red[v] = acc1;
    }
  }
}

// The divisions a transition may need (beta of the next step, alpha_l of the
// accepted one), computed speculatively in parallel lanes of warp 0 after the
// reduction: a GB300 FP64 division has a latency of several hundred cycles.
// Identical operands and operation to the serial form, so identical values.
__device__ __forceinline__ void precompute_divisions(const SolveState& S, const double* red, double* qd, int mixed) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    const bool step = S.pending == K_PA || S.pending == K_PF;
    double q = 0.0;
    if (lane < kMaxK) {
      if (step && lane <= S.nu) q = -red[1 + lane] / S.lpn2[lane];  // alpha_lane
    } else if (lane == kMaxK) {
      if (S.pending == K_INIT) q = -red[2] / red[3];  // first beta
      if (S.pending == K_PB || S.pending == K_RESTORE) q = -red[0] / red[1];  // next beta
    }
    if (mixed && step) {
      // The next direction's dots without forming it (mixed path, fused
      // step): L(p') = L(e) + sum_l alpha_l L(p^l) with the L(p^l) mutually
      // orthogonal and r' orthogonal to them (GCR), so
      //   <r', L(p')>    = <r', L(e)> = h,
      //   <L(p'), L(p')> = <L(e), L(e)> + sum_l alpha_l <L(e), L(p^l)> = q + sum_l alpha_l d_l.
      const double ad = lane < kMaxK && lane <= S.nu ? q * red[1 + lane] : 0.0;
      const double sum = warp_sum(ad);
      const double h = red[2 + S.nu], qq = red[3 + S.nu];
      const double den = qq + sum;
      // use the identities only while they keep three digits of <L(p'),L(p')>
      const bool ok = den > 1e-3 * qq && isfinite(den) && isfinite(h);
      if (lane == kMaxK + 1) q = ok ? -h / den : 0.0;  // next beta
      if (lane == kMaxK + 2) q = ok ? den : -1.0;      // <L(p'), L(p')>, or -1: form p' (PB)
    }
    qd[lane] = q;
  }
}

// ------------------------------------------------------------ transition
__device__ __forceinline__ int first_not2(int a, int b) {
  for (int i = 0; i < 3; ++i)
    if (i != a && i != b) return i;
  return 0;
}
__device__ __forceinline__ int first_not1(int a) { return a == 0 ? 1 : 0; }

template <typename T>
__device__ int new_slot(const SolveDev<T>& sd, const SolveState& N, int nu) {
  for (int s = 0; s < sd.k + 2; ++s) {
    bool used = (s == N.slotS);
    for (int l = 0; l <= nu; ++l) used = used || (N.slot[l] == s);
    if (!used) return s;
  }
  return 0;
}

// Partial sums reduced every round: the most any phase leaves (PA / PF: the
// norm, k dots and, on the mixed path, h and q; INIT: 4).
template <typename T>
__device__ __forceinline__ int part_values(const SolveDev<T>& sd) {
  const int n = sd.mixed ? sd.k + 3 : sd.k + 1;
  return n > 4 ? n : 4;
}

// Number of partial sums the phase `kind` leaves per tile.
__device__ __forceinline__ int part_count(int kind, int nu) {
  switch (kind) {
    case K_INIT: return 4;
    case K_PA:
    case K_PF: return 4 + nu;  // FP64 path: 2 + nu (no h, q)
    case K_PB:
    case K_RESTORE: return 2;
    case K_OUT: return 2;
    case K_FIN: return 1;
    default: return 0;
  }
}

// The per-solve state machine: consumes the reduced partial sums of the phase
// that ran last round (S.pending) and decides this round's phase.  Thread 0.
template <typename T>
__device__ __noinline__ void transition(const SolveDev<T>& sd, const SolveState& S, const double* red, const double* qd,
                                       SolveState& N, Ctx<T>& c) {
  // On entry N is a copy of S and c is zeroed (every pointer a phase may
  // test starts out null); the caller makes both copies block-wide.
  c.kind = K_NONE;
  c.nu = S.nu;
  c.t = S.step + 1;
  c.patch_step = S.step + 1;
  int dbuf = -1;       // OUT: phi buffer holding the inner solution
  int finbuf = -1;     // FIN: phi buffer holding the iterate to return
  bool to_out = false; // mixed: leave the inner solve
  bool to_fin = false;
  switch (S.pending) {
    case K_NONE:
      if (sd.mixed && sd.zero_guess) {
        // x0 = 0: r_out = R, so the first inner solve takes R as it is
        c.kind = K_INIT;
        c.zero_guess = 1;
        c.rin_R = 1;
        N.xzero = 1;
      } else if (sd.mixed) {
        c.kind = K_OUT;
        c.xsrc_user = 1;
        c.first = 1;
      } else {
        c.kind = K_INIT;
        if (sd.zero_guess) {
          c.zero_guess = 1;
          c.rin_R = 1;
        }
      }
      break;
    case K_OUT: {
      // mixed refinement: x' = x + d was formed, r_out = R - L64(x') reduced.
      // The paper's monotonicity test, applied to the FP64 outer residual,
      // rejects an update d that did not lower it (a flip in x or p of the
      // inner solve is invisible to the inner test but not to this one).
      const double nrm2_out = red[0];
      bool accept = true;
      if (S.first_out) {
        N.nrm2_R = red[1];
        N.thr2 = sd.tol2 * N.nrm2_R;
        N.first_out = 0;
        N.nrm2_0 = nrm2_out;
      } else if (sd.protect && !S.out_redo && !(nrm2_out < S.nrm2_out)) {
        accept = false;
      }
      N.outer = S.outer + 1;
      N.out_redo = 0;
      if (!accept) {
        N.fdet = S.fdet + 1;
        N.restarts = S.restarts + 1;
        if (S.ndetect < kMaxDetect) {
          N.detect_step[S.ndetect] = S.step;
          N.detect_ratio[S.ndetect] = nrm2_out / S.nrm2_out;
          N.ndetect = S.ndetect + 1;
        }
        N.out_rej = S.out_rej + 1;
        if (N.out_rej >= 3 || N.outer > sd.max_outer) {
          N.status = S.nrm2_out <= N.thr2 ? ST_CONVERGED : ST_NOT_CONVERGED;
          to_fin = true;
        } else {
          // recompute R_in and r_out for the kept x, then redo the inner solve
          N.out_redo = 1;
          c.kind = K_OUT;
          c.d = nullptr;
          c.xsrc = S.xzero ? nullptr : sd.xbuf[S.xcur];
          c.xdst = sd.xbuf[S.xcur ^ 1];
        }
        break;
      }
      N.out_rej = 0;
      N.xcur = S.xcur ^ 1;
      N.xzero = 0;
      N.nrm2_out = nrm2_out;
      if (N.nrm2_R == 0.0) {
        N.status = ST_CONVERGED;
        to_fin = true;
      } else if (nrm2_out <= N.thr2) {
        N.status = ST_CONVERGED;
        to_fin = true;
      } else if (N.outer > sd.max_outer || S.step >= sd.max_steps) {
        N.status = ST_NOT_CONVERGED;
        to_fin = true;
      } else {
        const double a = sd.inner_tol2 * nrm2_out, b = 0.25 * N.thr2;
        N.thr2_in = a > b ? a : b;
        N.phiC = 0;
        N.rC = 0;
        N.slot[0] = 0;
        N.nu = 0;
        N.stag = 0;
        c.kind = K_INIT;
        c.zero_guess = 1;
      }
      break;
    }
    case K_INIT: {
      double thr2;
      if (!sd.mixed) {
        N.nrm2_R = red[1];
        N.thr2 = sd.tol2 * N.nrm2_R;
        N.nrm2_0 = red[0];
        thr2 = N.thr2;
      } else if (S.first_out) {
        // zero initial guess: this INIT took R itself, and its FP64 ||R||^2
        // stands for the first OUT's (r_out = R)
        N.nrm2_R = red[1];
        N.thr2 = sd.tol2 * N.nrm2_R;
        N.first_out = 0;
        N.nrm2_0 = N.nrm2_R;
        N.nrm2_out = N.nrm2_R;
        N.outer = S.outer + 1;
        const double a = sd.inner_tol2 * N.nrm2_R, b = 0.25 * N.thr2;
        N.thr2_in = a > b ? a : b;
        thr2 = N.thr2_in;
        if (N.nrm2_R == 0.0) {  // R = 0: x = 0 is the solution
          N.status = ST_CONVERGED;
          to_fin = true;
          break;
        }
      } else {
        thr2 = S.thr2_in;
      }
      N.nrm2_prev = red[0];
      N.nrm2_last = red[0];
      N.phiS = N.phiC;
      N.rS = N.rC;
      N.slotS = N.slot[0];
      N.nrm2_S = red[0];
      N.patched = count_faults(sd, S.step + 1, kStateVecs) > 0;
      N.patch_step = S.step + 1;
      N.nu = 0;
      if (!sd.mixed && N.nrm2_R == 0.0) {
        N.status = ST_CONVERGED;
        c.finzero = 1;
        to_fin = true;
      } else if (red[0] <= thr2) {
        if (!sd.mixed) {
          N.status = ST_CONVERGED;
          finbuf = N.phiC;
          c.patched = N.patched;
          c.patch_step = N.patch_step;
          to_fin = true;
        } else {
          to_out = true;  // nothing to add
        }
      } else if (S.step >= sd.max_steps) {
        if (!sd.mixed) {
          N.status = ST_NOT_CONVERGED;
          finbuf = N.phiC;
          c.patched = N.patched;
          c.patch_step = N.patch_step;
          to_fin = true;
        } else {
          to_out = true;
        }
      } else {
        N.finj += count_faults(sd, S.step + 1, kStateVecs);
        N.beta = qd[kMaxK];  // -red[2] / red[3]
        N.lpn2[0] = red[3];
        c.kind = K_PA;
      }
      break;
    }
    case K_PA:
    case K_PF: {
      const long long t = S.step + 1;
      N.step = t;
      const double nrm2 = red[0];
      N.nrm2_last = nrm2;
      const double thr2 = sd.mixed ? S.thr2_in : S.thr2;
      if (nrm2 <= thr2) {  // exit test first (Algorithm 1)
        if (!sd.mixed) {
          N.status = ST_CONVERGED;
          finbuf = S.phiW;
          to_fin = true;
        } else {
          dbuf = S.phiW;
          to_out = true;
        }
      } else if (sd.protect && !(nrm2 < S.nrm2_prev)) {  // fault test (Algorithm 1, red part)
        N.fdet = S.fdet + 1;
        N.restarts = S.restarts + 1;
        if (S.ndetect < kMaxDetect) {
          N.detect_step[S.ndetect] = t;
          N.detect_ratio[S.ndetect] = nrm2 / S.nrm2_prev;
          N.ndetect = S.ndetect + 1;
        }
        N.stag = S.stag + 1;
        if (t >= sd.max_steps) {
          if (!sd.mixed) {
            N.status = ST_NOT_CONVERGED;
            finbuf = S.phiS;
            c.patched = S.patched;
            c.patch_step = S.patch_step;
            to_fin = true;
          } else {
            dbuf = S.patched ? -1 : S.phiS;
            to_out = true;
          }
        } else if (sd.mixed && N.stag >= 2) {
          // mixed only: a repeated rejection without progress means the FP32
          // inner iteration has stagnated; hand the backup to the refinement
          dbuf = S.patched ? -1 : S.phiS;
          to_out = true;
        } else {
          c.kind = K_RESTORE;
          N.phiC = first_not1(S.phiS);
          N.rC = first_not1(S.rS);
          N.slot[0] = (S.slotS == 0) ? 1 : 0;
          N.nu = 0;
          N.nrm2_prev = S.nrm2_S;
          c.t = t + 1;
        }
      } else {  // accepted
        N.stag = 0;
        N.finj = S.finj + count_faults(sd, t, 1u << V_E);
        N.lossev = S.lossev + count_losses(sd, t);
        if (S.nu == 0) {  // ^* <- ^0
          N.phiS = S.phiC;
          N.rS = S.rC;
          N.slotS = S.slot[0];
          N.nrm2_S = S.nrm2_prev;
          N.patched = 0;
        }
        N.nrm2_prev = nrm2;
        N.phiC = S.phiW;
        N.rC = S.rW;
        if (t >= sd.max_steps) {
          if (!sd.mixed) {
            N.status = ST_NOT_CONVERGED;
            finbuf = N.phiC;
            to_fin = true;
          } else {
            dbuf = N.phiC;
            to_out = true;
          }
        } else {
          c.kind = K_PB;
          c.nu = S.nu;
          c.t = t + 1;
          const int ns = new_slot(sd, N, S.nu);
          N.slot[S.nu + 1] = ns;
          if (S.nu + 1 == sd.k) {
            N.slot[0] = ns;
            N.nu = 0;
            N.cycles = S.cycles + 1;
          } else {
            N.nu = S.nu + 1;
          }
          c.pnew = sd.p[ns];
          c.lpnew = sd.Lp[ns];
          if (sd.mixed && qd[kMaxK + 2] > 0.0) {
            // mixed path: form p' and take step t + 1 with it in one round
            // (PF), beta and <L(p'), L(p')> from the identities
            c.kind = K_PF;
            c.nuo = S.nu;
            N.beta = qd[kMaxK + 1];
            N.lpn2[N.nu] = qd[kMaxK + 2];
            N.finj += count_faults(sd, t + 1, kStateVecs);
          }
        }
      }
      break;
    }
    case K_PB:
    case K_RESTORE:
      N.finj = S.finj + count_faults(sd, S.step + 1, kStateVecs);
      N.beta = qd[kMaxK];  // -red[0] / red[1]
      N.lpn2[S.nu] = red[1];
      c.kind = K_PA;
      break;
    case K_FIN:
      N.res_true2 = sd.mixed ? S.nrm2_out : red[0];
      N.active = 0;
      c.kind = K_NONE;
      break;
    default:
      N.active = 0;
      break;
  }
  if (to_out) {
    c.kind = K_OUT;
    c.d = dbuf >= 0 ? sd.phi[dbuf] : nullptr;
  }
  if (to_fin) {
    c.kind = K_FIN;
    if (!sd.mixed) {
      c.finsrc = finbuf >= 0 ? sd.phi[finbuf] : nullptr;
      if (finbuf < 0) c.finzero = 1;
    }
  }
  // pointers for this round's phase
  if (c.kind == K_PA || c.kind == K_PF) {
    N.phiW = first_not2(N.phiC, N.phiS);
    N.rW = first_not2(N.rC, N.rS);
    c.nu = N.nu;
    c.t = N.step + 1;
    c.beta = (T)N.beta;
    c.phiC = sd.phi[N.phiC];
    c.phiW = sd.phi[N.phiW];
    c.rC = sd.r[N.rC];
    c.rW = sd.r[N.rW];
    c.pnu = sd.p[N.slot[N.nu]];
    c.lpnu = sd.Lp[N.slot[N.nu]];
    if (c.kind == K_PF) {
      c.eR = sd.e[S.ecur];
      c.LeR = sd.Le[S.ecur];
    }
    N.ecur = sd.mixed ? (S.ecur ^ 1) : 0;
    c.eW = sd.e[N.ecur];
    c.LeW = sd.Le[N.ecur];
  } else if (c.kind == K_PB) {
    c.phiCw = sd.phi[N.phiC];
    c.rCw = sd.r[N.rC];
    c.eR = sd.e[S.ecur];
    c.LeR = sd.Le[S.ecur];
  } else if (c.kind == K_RESTORE) {
    c.phiS = sd.phi[S.phiS];
    c.rS = sd.r[S.rS];
    c.pS = sd.p[S.slotS];
    c.lpS = sd.Lp[S.slotS];
    c.phiT = sd.phi[N.phiC];
    c.rT = sd.r[N.rC];
    c.pT = sd.p[N.slot[0]];
    c.lpT = sd.Lp[N.slot[0]];
    c.patched = S.patched;
    c.patch_step = S.patch_step;
  } else if (c.kind == K_INIT) {
    c.t = N.step + 1;
    c.phiW = sd.phi[N.phiC];
    c.rW = sd.r[N.rC];
    c.pnew = sd.p[N.slot[0]];
    c.lpnew = sd.Lp[N.slot[0]];
  } else if (c.kind == K_OUT && !N.out_redo) {
    c.xsrc = c.xsrc_user ? sd.x0 : (N.xzero ? nullptr : sd.xbuf[S.xcur]);
    c.xdst = sd.xbuf[S.xcur ^ 1];
  } else if (c.kind == K_FIN) {
    if (sd.mixed) c.xsrc = N.xzero ? nullptr : sd.xbuf[N.xcur];
  }
  N.pending = c.kind;
  if (c.kind == K_NONE) N.active = 0;
}

// The per-direction entries of the context the transition chose (alpha and
// the p / L(p) slot pointers), one direction per thread: threads 0..kMaxK-1
// of the block, after the transition.
template <typename T>
__device__ __forceinline__ void fill_directions(const SolveDev<T>& sd, const SolveState& S, const SolveState& N,
                                                const double* qd, Ctx<T>& c) {
  const int l = threadIdx.x;
  if (l >= kMaxK) return;
  if (c.kind == K_PA || c.kind == K_PF) {
    if (l <= N.nu) c.lp[l] = sd.Lp[N.slot[l]];
    if (c.kind == K_PF && l <= S.nu) {
      c.pp[l] = sd.p[S.slot[l]];
      c.lo[l] = sd.Lp[S.slot[l]];
      c.alpha[l] = (T)qd[l];  // -<L(e), L(p^l)> / <L(p^l), L(p^l)>
    }
  } else if (c.kind == K_PB && l <= S.nu) {
    c.pp[l] = sd.p[S.slot[l]];
    c.lp[l] = sd.Lp[S.slot[l]];
    c.alpha[l] = (T)qd[l];
  }
}

// ------------------------------------------------------------ phases
struct PhaseSmem {
  int cs_solve, cs_tile;  // (solve, tile) whose line-solve constants sit in shared memory
  FlipEnt fl[kMaxFaults];
  FlipEnt pt[kMaxFaults];
  int nfl, npt;
  CtaRed cr;
  unsigned long long sub[3];  // sub-phase timestamps (trace only)
  int tracing;
};
__device__ __forceinline__ void sub_mark(PhaseSmem& ps, int q) {
  if (ps.tracing && threadIdx.x == 0) ps.sub[q] = globaltimer();
}

// Line-solve constants of rows [h0, h1) staged into shared memory by
// asynchronous 16-byte copies (cp.async; waited for before the solves): three
// arrays, rows contiguous.  FP32 path: chunk layout c, 1/w, z (32 C per row);
// FP64 path: natural-layout factors l, 1/w, u (nlon per row).
template <typename T>
__device__ __forceinline__ long long consts_per_row(const SolveDev<T>& sd) {
  if constexpr (sizeof(T) == 8)
    return sd.lchunk ? 32LL * sd.C : sd.nlon;
  else
    return 32LL * sd.C;
}
// GL (FP64 wide-row instance): a solve whose factors stay in global memory
// stages none.
template <typename T, bool GL = false>
__device__ __forceinline__ void stage_line_consts(const SolveDev<T>& sd, int h0, int h1, T* cs) {
  if (sd.precond != PC_LINE) return;
  if constexpr (GL && sizeof(T) == 8) {
    if (sd.cs_global) return;  // read from global memory by the row solves
  }
  const long long per = consts_per_row(sd);
  const int nrows = h1 - h0;
  const long long nel = (long long)nrows * per;
  const T* src[3];
  if constexpr (sizeof(T) == 8) {
    src[0] = sd.lchunk ? sd.lcc : sd.lc;
    src[1] = sd.lchunk ? sd.lwc : sd.lw;
    src[2] = sd.lchunk ? sd.lzc : sd.lu;
  } else {
    src[0] = sd.lc;
    src[1] = sd.lw;
    src[2] = sd.lz;
  }
  constexpr int W = V16<T>::W;
  if ((per % W) == 0) {
    const long long nv = nel / W;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T* g = src[a] + (long long)h0 * per;
      T* d = cs + (long long)a * nel;
      for (long long q = threadIdx.x; q < nv; q += kThreads) cp_async16(d + q * W, g + q * W);
    }
    cp_async_commit();
  } else {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const T* g = src[a] + (long long)h0 * per;
      T* d = cs + (long long)a * nel;
      for (long long q = threadIdx.x; q < nel; q += kThreads) d[q] = __ldg(g + q);
    }
  }
}
template <typename T>
__device__ __forceinline__ LineConsts<T> staged_consts(const SolveDev<T>& sd, const T* cs, int nrows, int r) {
  const long long per = consts_per_row(sd);
  return LineConsts<T>{cs + (long long)r * per, cs + ((long long)nrows + r) * per, cs + (2LL * nrows + r) * per};
}

// The FP64 line solve of a tile whose factors stay in global memory (wide
// rows): the same steps as the staged form in precond_tile, with the tile's
// factor rows first asked of L2 (rows of 256+ columns: the chunked solve,
// one warp per row, reading the chunk-layout factors from global memory).  ring: kRingStride doubles of shared memory
// per row for the chains' factor rings.  Its own function, so that the staged
// form's code is the same as without it.
static __device__ __noinline__ void precond_tile_gl(const SolveDev<double>& sd, int h0, int nrows, double* sm,
                                                    int stride, double* ring) {
  const int n = sd.nlon, m = n - 1;
  if (sd.lchunk) {
    // rows of 256+ columns: the chunked solve, one warp per row, its factors
    // read from global memory in the chunk layout (first asked of L2)
    const long long per = 32LL * sd.C, b0 = (long long)h0 * per, l0 = (long long)nrows * per;
    for (long long q = 16LL * threadIdx.x; q < l0; q += 16LL * kThreads) {
      prefetch_l2(sd.lcc + b0 + q);
      prefetch_l2(sd.lwc + b0 + q);
      prefetch_l2(sd.lzc + b0 + q);
    }
    for (int jr = threadIdx.x >> 5; jr < nrows; jr += kWarps)
      line_solve_row<double, true>(sd, h0 + jr, sm + jr * stride,
                                   LineConsts<double>{sd.lcc + b0 + jr * per, sd.lwc + b0 + jr * per,
                                                      sd.lzc + b0 + jr * per});
    return;
  }
  const long long base = (long long)h0 * n, len = (long long)nrows * n;
  for (long long q = 16LL * threadIdx.x; q < len; q += 16LL * kThreads) {  // 128-byte lines
    prefetch_l2(sd.lc + base + q);
    prefetch_l2(sd.lw + base + q);
    prefetch_l2(sd.lu + base + q);
  }
  // the rows' chains spread over up to four warps (one per SM sub-partition,
  // each with its own FP64 unit): row w + nw q in lane q of warp w
  const int nw = min(nrows, 4), wq = threadIdx.x >> 5, lq = threadIdx.x & 31;
  const int jc = wq < nw ? wq + nw * lq : nrows;  // this thread's row, if any
  if (jc < nrows) line_solve_fwd_gl(n, sm + jc * stride, sd.lc + base + (long long)jc * n, ring + jc * kRingStride);
  __syncthreads();
  // the backward step's products g_i winv_i, all rows at once (row by row,
  // each thread's loads of a group issued together)
  constexpr int kU = 8;
  for (int jr = 0; jr < nrows; ++jr) {
    const unsigned rb = smem_addr(sm + jr * stride);
    const double* w = sd.lw + base + (long long)jr * n;
    for (int i0 = threadIdx.x; i0 < m; i0 += kU * kThreads) {
      double wv[kU];
#pragma unroll
      for (int q = 0; q < kU; ++q) wv[q] = i0 + q * kThreads < m ? __ldg(w + i0 + q * kThreads) : 0.0;
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        const int i = i0 + q * kThreads;
        if (i < m) {
          const unsigned a = rb + 8u * (unsigned)sk(i);
          sts(a, lds<double>(a) * wv[q]);
        }
      }
    }
  }
  __syncthreads();
  if (jc < nrows)
    line_solve_bwd_gl(sd, h0 + jc, sm + jc * stride, sd.lu + base + (long long)jc * n, ring + jc * kRingStride);
  __syncthreads();
  // bordering, x_i = y_i - x_{n-1} z_i, all rows at once
  for (int jr = 0; jr < nrows; ++jr) {
    const unsigned rb = smem_addr(sm + jr * stride);
    const double* z = sd.lz + base + (long long)jr * n;
    const double xl = lds<double>(rb + 8u * (unsigned)sk(n - 1));
    for (int i0 = threadIdx.x; i0 < m; i0 += kU * kThreads) {
      double zv[kU];
#pragma unroll
      for (int q = 0; q < kU; ++q) zv[q] = i0 + q * kThreads < m ? __ldg(z + i0 + q * kThreads) : 0.0;
#pragma unroll
      for (int q = 0; q < kU; ++q) {
        const int i = i0 + q * kThreads;
        if (i < m) {
          const unsigned a = rb + 8u * (unsigned)sk(i);
          sts(a, lds<double>(a) - xl * zv[q]);
        }
      }
    }
  }
}

// The preconditioner on the nrows rows of a tile staged in shared memory.
// FP32 line solve, FP64 line solve on rows of 256+ columns and the pointwise
// preconditioners: one warp per row.  FP64 line solve on narrower rows: one
// lane per row, the rows side by side in the first warp(s).
// Each row's solve is the oracle's serial elimination, a chain of dependent
// FP64 operations, and GB300 issues an FP64 warp instruction at the same cost
// whatever the number of active lanes (measured: 64 cycles per dependent FMA
// for 1 to 32 lanes of one warp, 152 with eight warps on the SM), so rows
// side by side in lanes cost one row's instructions instead of one per row.
// GROUPS (mixed path, kernel instance with split rounds) and `groups` (the
// first pass of a split round): a tile with at most half as many rows as
// warps solves each row with a group of 2, 4 or 8 warps.  One-pass rounds
// keep one warp per row in every instance, so a one-pass solve gives the
// same result in a launch with split solves as alone.
template <typename T, bool GROUPS = false, bool GL = false>
__device__ __forceinline__ void precond_tile(const SolveDev<T>& sd, int h0, int nrows, T* sm, int stride, const T* cs,
                                             bool groups = false) {
  if constexpr (sizeof(T) == 8) {
    if (sd.precond == PC_LINE) {
      if constexpr (GL) {
        if (sd.cs_global) {
          precond_tile_gl(sd, h0, nrows, sm, stride, const_cast<T*>(cs));
          return;
        }
      }
      if (sd.lchunk) {
        // one warp per row: the chunked solve of the FP32 path in FP64 (the
        // row's recurrences as 32 per-lane chunks joined by an exact scan of
        // their affine maps)
        const int warp = threadIdx.x >> 5;
        for (int jr = warp; jr < nrows; jr += kWarps)
          line_solve_row<double>(sd, h0 + jr, sm + jr * stride, staged_consts(sd, cs, nrows, jr));
        return;
      }
      const int n = sd.nlon, m = n - 1;
      for (int jr = threadIdx.x; jr < nrows; jr += kThreads)
        line_solve_fwd_sh(n, sm + jr * stride, staged_consts(sd, cs, nrows, jr).cb);
      __syncthreads();
      // the backward step's products g_i winv_i, all rows at once
      for (int idx = threadIdx.x; idx < nrows * m; idx += kThreads) {
        const int jr = idx / m, i = idx - jr * m;
        T* row = sm + jr * stride;
        row[sk(i)] = row[sk(i)] * staged_consts(sd, cs, nrows, jr).cw[i];
      }
      __syncthreads();
      for (int jr = threadIdx.x; jr < nrows; jr += kThreads)
        line_solve_bwd_sh(sd, h0 + jr, sm + jr * stride, staged_consts(sd, cs, nrows, jr).cz);
      __syncthreads();
      // bordering, x_i = y_i - x_{n-1} z_i, all rows at once
      for (int idx = threadIdx.x; idx < nrows * m; idx += kThreads) {
        const int jr = idx / m, i = idx - jr * m;
        T* row = sm + jr * stride;
        row[sk(i)] = row[sk(i)] - row[sk(n - 1)] * __ldg(sd.lz + (long long)(h0 + jr) * n + i);
      }
      return;
    }
  }
  const int warp = threadIdx.x >> 5;
  if constexpr (GROUPS && sizeof(T) == 4) {
    if (groups && sd.precond == PC_LINE && 2 * nrows <= kWarps) {
      __shared__ float maps[kWarps * 64];  // per group: 2 x 32 x G
      auto run = [&](auto gtag) {
        constexpr int G = decltype(gtag)::value;
        const int grp = warp / G;
        if (grp < nrows)
          line_solve_row_group<G>(sd, h0 + grp, sm + grp * stride, staged_consts(sd, cs, nrows, grp),
                                  maps + grp * 64 * G, 1 + grp);
      };
      const int C = sd.C;
      if (8 * nrows <= kWarps && C % 64 == 0) {
        run(std::integral_constant<int, 8>());
        return;
      }
      if (4 * nrows <= kWarps && C % 32 == 0) {
        run(std::integral_constant<int, 4>());
        return;
      }
      if (C % 16 == 0) {
        run(std::integral_constant<int, 2>());
        return;
      }
    }
  }
  for (int jr = warp; jr < nrows; jr += kWarps) precond_row(sd, h0 + jr, sm + jr * stride, staged_consts(sd, cs, nrows, jr));
}

// Row-tile halo rows: [h0, h1) = [j0-1, j1+1) clipped to the sphere.
struct RowTile {
  int j0, j1, h0, h1;
};
__device__ __forceinline__ RowTile row_tile(int nlat, int nt, int tau) {
  RowTile t;
  t.j0 = row_start(nlat, nt, tau);
  t.j1 = row_start(nlat, nt, tau + 1);
  t.h0 = t.j0 > 0 ? t.j0 - 1 : 0;
  t.h1 = t.j1 < nlat ? t.j1 + 1 : nlat;
  return t;
}

// Stencil on shared-memory rows (row r of the tile at sm + r*stride, rows
// [h0, h1)) for own row j, column i.
template <typename T>
__device__ __forceinline__ T stencil_smem(const SolveDev<T>& sd, const T* sm, int stride, int h0, int j, int i) {
  const int nlon = sd.nlon, nlat = sd.nlat;
  const T* row = sm + (j - h0) * stride;
  const int ie = (i + 1 == nlon) ? 0 : i + 1;
  const int iw = (i == 0) ? nlon - 1 : i - 1;
  const long long g = (long long)j * nlon + i;
  const bool hasN = j < nlat - 1, hasS = j > 0;
  const T v = row[sk(i)];
  const T vn = hasN ? row[stride + sk(i)] : T(0);
  const T vs = hasS ? row[-stride + sk(i)] : T(0);
  return stencil_op<T>(sd.oracle_order, v, row[sk(ie)], row[sk(iw)], vn, vs, __ldg(sd.Tx + g),
                       __ldg(sd.Tx + (long long)j * nlon + iw), hasN ? __ldg(sd.Ty + g) : T(0),
                       hasS ? __ldg(sd.Ty + g - nlon) : T(0), __ldg(sd.muA + j), hasN, hasS);
}

// Stencil on a global-memory field (initialisation / final residual; the
// operator entry point, always in the oracle's form).
template <typename V>
__device__ __forceinline__ V stencil_global(const V* x, const V* Tx, const V* Ty, const V* muA, int nlon, int nlat,
                                            int j, int i, int oracle_order = 1) {
  const int ie = (i + 1 == nlon) ? 0 : i + 1;
  const int iw = (i == 0) ? nlon - 1 : i - 1;
  const long long g = (long long)j * nlon + i;
  const bool hasN = j < nlat - 1, hasS = j > 0;
  const V v = ldcg(x + g);
  const V vn = hasN ? ldcg(x + g + nlon) : V(0);
  const V vs = hasS ? ldcg(x + g - nlon) : V(0);
  return stencil_op<V>(oracle_order, v, ldcg(x + (long long)j * nlon + ie), ldcg(x + (long long)j * nlon + iw), vn,
                       vs, __ldg(Tx + g), __ldg(Tx + (long long)j * nlon + iw), hasN ? __ldg(Ty + g) : V(0),
                       hasS ? __ldg(Ty + g - nlon) : V(0), __ldg(muA + j), hasN, hasS);
}

// Element (j, i) of a row-tile loop over 16-byte vectors: flat index ->
// (row, first column).
struct RowVec {
  int j, i;
  long long g;
};
__device__ __forceinline__ RowVec row_vec(int idx, int nvr, int j0, int nlon, int W) {
  RowVec r;
  const int jr = idx / nvr;
  r.j = j0 + jr;
  r.i = (idx - jr * nvr) * W;
  r.g = (long long)r.j * nlon + r.i;
  return r;
}

// Rows [h0, h1) of a vector written by other CTAs this round into the
// shared-memory row layout (L2 loads, four 16-byte loads per thread in flight).
template <typename T>
__device__ __forceinline__ void stage_rows(const T* src, int h0, int h1, int nlon, T* sm, int stride) {
  constexpr int W = V16<T>::W, U = 4;
  if (nlon % W == 0) {
    const int nvr = nlon / W, total = (h1 - h0) * nvr;
    for (int b0 = threadIdx.x; b0 < total; b0 += U * kThreads) {
      V16<T> v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = b0 + u * kThreads;
        if (idx < total) v[u] = ldv(src + (long long)h0 * nlon + (long long)idx * W);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = b0 + u * kThreads;
        if (idx < total) {
          const int jr = idx / nvr, i = (idx - jr * nvr) * W;
          T* row = sm + jr * stride;
#pragma unroll
          for (int w = 0; w < W; ++w) row[sk(i + w)] = v[u].v[w];
        }
      }
    }
  } else {
    for (int j = h0; j < h1; ++j) {
      T* row = sm + (j - h0) * stride;
      for (int i = threadIdx.x; i < nlon; i += kThreads) row[sk(i)] = ldcg(src + (long long)j * nlon + i);
    }
  }
}
// Rows [h0, h1) of the shared-memory row layout out to a vector.
template <typename T>
__device__ __forceinline__ void store_rows(T* dst, int h0, int h1, int nlon, const T* sm, int stride) {
  constexpr int W = V16<T>::W;
  if (nlon % W == 0) {
    const int nvr = nlon / W, total = (h1 - h0) * nvr;
    for (int idx = threadIdx.x; idx < total; idx += kThreads) {
      const int jr = idx / nvr, i = (idx - jr * nvr) * W;
      const T* row = sm + jr * stride;
      V16<T> v;
#pragma unroll
      for (int w = 0; w < W; ++w) v.v[w] = row[sk(i + w)];
      stv(dst + (long long)h0 * nlon + (long long)idx * W, v);
    }
  } else {
    for (int j = h0; j < h1; ++j) {
      const T* row = sm + (j - h0) * stride;
      for (int i = threadIdx.x; i < nlon; i += kThreads) dst[(long long)j * nlon + i] = row[sk(i)];
    }
  }
}

// The data-loss events of step t (Section 3) on the e rows [h0, h1) staged in
// shared memory: every thread takes flips i = 1 + threadIdx.x, ... of each
// event and XORs those that land in the tile (atomically: two flips may hit
// the same word, and XOR makes their order irrelevant).
template <typename T>
__device__ __forceinline__ void apply_losses(const SolveDev<T>& sd, long long t, int h0, int h1, T* sm, int stride) {
  using U = typename std::conditional<sizeof(T) == 8, unsigned long long, unsigned int>::type;
  constexpr unsigned kBits = 8 * sizeof(T);
  const int nlon = sd.nlon;
  const long long g0 = (long long)h0 * nlon, g1 = (long long)h1 * nlon;
  for (int q = 0; q < sd.nlosses; ++q) {
    const LossEv ev = sd.losses[q];
    if (ev.step != t) continue;
    const long long b0 = (long long)ev.rank * sd.N / ev.nranks, b1 = (long long)(ev.rank + 1) * sd.N / ev.nranks;
    const long long len = b1 - b0;
    if (len <= 0 || b1 <= g0 || b0 >= g1) continue;
    for (long long i = 1 + threadIdx.x; i <= ev.count; i += kThreads) {
      const unsigned long long z = splitmix64_at(ev.seed, (unsigned long long)i);
      const long long g = b0 + (long long)(z % (unsigned long long)len);
      if (g < g0 || g >= g1) continue;
      const int j = (int)(g / nlon), col = (int)(g - (long long)j * nlon);
      U* w = reinterpret_cast<U*>(sm + (j - h0) * stride + sk(col));
      atomicXor(w, (U)1 << (unsigned)((z >> 32) % kBits));
    }
  }
}

// The parts of a step phase (PA, PF), inlined into the one-pass phase and
// into the two passes of a split round.  Rows [rt.h0, rt.h1) are staged in
// shared memory (own rows [rt.j0, rt.j1) and, in one-pass rounds, a halo row
// each side).
// (1) The axpy: r' (and, fused, the new direction) into the staged rows; the
// state vectors of the own rows written; an += ||r'||^2 over own rows.
template <typename T, int KB, bool FUSED>
__device__ __forceinline__ void step_axpy(const SolveDev<T>& sd, const Ctx<T>& c, const RowTile& rt, T* sm,
                                          PhaseSmem& ps, Acc<T>& an) {
  constexpr int W = V16<T>::W;
  constexpr int U = 2;
  const int nlon = sd.nlon, nlat = sd.nlat, stride = row_stride(nlon);
  const int nrows = rt.h1 - rt.h0;
  const T beta = c.beta;
  if constexpr (FUSED) {
    // p' = e + sum_l alpha_l p^l, L(p') = L(e) + sum_l alpha_l L(p^l) (l in
    // increasing order, one fma per term, as PB), then the flips of the
    // start of this step (x, r, p', L(p')), then r'' = r' + beta L(p') and
    // phi'' = phi' + beta p'.  Halo rows form only L(p') and r''.
    __syncthreads();
    const int nfl = ps.nfl;
    auto fuse = [&](long long g, T& ln, T& rr, T& pn, T& ph, bool own) {
      if (nfl) {
        rr = apply_flips(rr, g, V_R, nfl, ps.fl);
        ln = apply_flips(ln, g, V_AP, nfl, ps.fl);
        if (own) {
          ph = apply_flips(ph, g, V_X, nfl, ps.fl);
          pn = apply_flips(pn, g, V_P, nfl, ps.fl);
        }
      }
    };
    if (nlon % W == 0) {
      const int nvr = nlon / W, total = nrows * nvr;
      for (int idx = threadIdx.x; idx < total; idx += kThreads) {
        const RowVec rv = row_vec(idx, nvr, rt.h0, nlon, W);
        const bool own = rv.j >= rt.j0 && rv.j < rt.j1;
        V16<T> ln = ldv(c.LeR + rv.g), rr = ldv(c.rC + rv.g), pn, ph;
#pragma unroll
        for (int w = 0; w < W; ++w) pn.v[w] = ph.v[w] = T(0);
        if (own) {
          pn = ldv(c.eR + rv.g);
          ph = ldv(c.phiC + rv.g);
        }
#pragma unroll
        for (int l = 0; l < KB; ++l)
          if (l <= c.nuo) {
            const T al = c.alpha[l];
            const V16<T> ll = ldv(c.lo[l] + rv.g);
#pragma unroll
            for (int w = 0; w < W; ++w) ln.v[w] = tfma(al, ll.v[w], ln.v[w]);
            if (own) {
              const V16<T> pl = ldv(c.pp[l] + rv.g);
#pragma unroll
              for (int w = 0; w < W; ++w) pn.v[w] = tfma(al, pl.v[w], pn.v[w]);
            }
          }
#pragma unroll
        for (int w = 0; w < W; ++w) fuse(rv.g + w, ln.v[w], rr.v[w], pn.v[w], ph.v[w], own);
        T* row = sm + (rv.j - rt.h0) * stride;
        V16<T> rn, fn;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          rn.v[w] = tfma(beta, ln.v[w], rr.v[w]);
          row[sk(rv.i + w)] = rn.v[w];
        }
        if (own) {
#pragma unroll
          for (int w = 0; w < W; ++w) {
            fn.v[w] = tfma(beta, pn.v[w], ph.v[w]);
            an.add(rn.v[w], rn.v[w]);
          }
          stv(c.pnew + rv.g, pn);
          stv(c.lpnew + rv.g, ln);
          stv(c.rW + rv.g, rn);
          stv(c.phiW + rv.g, fn);
        }
      }
    } else {
      for (int j = rt.h0; j < rt.h1; ++j) {
        const bool own = (j >= rt.j0 && j < rt.j1);
        T* row = sm + (j - rt.h0) * stride;
        const long long base = (long long)j * nlon;
        for (int i = threadIdx.x; i < nlon; i += kThreads) {
          const long long g = base + i;
          T ln = ldcg(c.LeR + g), rr = ldcg(c.rC + g), pn = T(0), ph = T(0);
          if (own) {
            pn = ldcg(c.eR + g);
            ph = ldcg(c.phiC + g);
          }
          for (int l = 0; l < KB; ++l)
            if (l <= c.nuo) {
              ln = tfma(c.alpha[l], ldcg(c.lo[l] + g), ln);
              if (own) pn = tfma(c.alpha[l], ldcg(c.pp[l] + g), pn);
            }
          fuse(g, ln, rr, pn, ph, own);
          const T rn = tfma(beta, ln, rr);
          row[sk(i)] = rn;
          if (own) {
            c.pnew[g] = pn;
            c.lpnew[g] = ln;
            c.rW[g] = rn;
            c.phiW[g] = tfma(beta, pn, ph);
            an.add(rn, rn);
          }
        }
      }
    }
  } else if (nlon % W == 0) {
    const int nvr = nlon / W, total = nrows * nvr;
    for (int b0 = threadIdx.x; b0 < total; b0 += U * kThreads) {
      V16<T> lp[U], rr[U], pv[U], ph[U];
      RowVec rv[U];
      bool ok[U], own[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int idx = b0 + u * kThreads;
        ok[u] = idx < total;
        if (ok[u]) {
          rv[u] = row_vec(idx, nvr, rt.h0, nlon, W);
          own[u] = rv[u].j >= rt.j0 && rv[u].j < rt.j1;
          lp[u] = ldv(c.lpnu + rv[u].g);
          rr[u] = ldv(c.rC + rv[u].g);
          if (own[u]) {
            pv[u] = ldv(c.pnu + rv[u].g);
            ph[u] = ldv(c.phiC + rv[u].g);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!ok[u]) continue;
        V16<T> rn, fn;
        T* row = sm + (rv[u].j - rt.h0) * stride;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          rn.v[w] = tfma(beta, lp[u].v[w], rr[u].v[w]);
          row[sk(rv[u].i + w)] = rn.v[w];
        }
        if (own[u]) {
#pragma unroll
          for (int w = 0; w < W; ++w) {
            fn.v[w] = tfma(beta, pv[u].v[w], ph[u].v[w]);
            an.add(rn.v[w], rn.v[w]);
          }
          stv(c.rW + rv[u].g, rn);
          stv(c.phiW + rv[u].g, fn);
        }
      }
    }
  } else {
    for (int j = rt.h0; j < rt.h1; ++j) {
      const bool own = (j >= rt.j0 && j < rt.j1);
      T* row = sm + (j - rt.h0) * stride;
      const long long base = (long long)j * nlon;
      for (int i = threadIdx.x; i < nlon; i += kThreads) {
        const long long g = base + i;
        const T r1 = tfma(beta, ldcg(c.lpnu + g), ldcg(c.rC + g));
        row[sk(i)] = r1;
        if (own) {
          c.rW[g] = r1;
          c.phiW[g] = tfma(beta, ldcg(c.pnu + g), ldcg(c.phiC + g));
          an.add(r1, r1);
        }
      }
    }
  }
}
// (2) e = P^-1 r' on the staged rows, then the e-site flips and data-loss
// events of the step.
template <typename T, bool GROUPS = false, bool GL = false>
__device__ __forceinline__ void step_precond(const SolveDev<T>& sd, const Ctx<T>& c, const RowTile& rt, T* sm,
                                             const T* cs, PhaseSmem& ps, bool groups = false) {
  const int nlon = sd.nlon, stride = row_stride(nlon);
  const int nrows = rt.h1 - rt.h0;
  cp_async_wait_all();
  __syncthreads();
  sub_mark(ps, 0);
  precond_tile<T, GROUPS, GL>(sd, rt.h0, nrows, sm, stride, cs, groups);
  __syncthreads();
  sub_mark(ps, 1);
  if (threadIdx.x == 0) {
    for (int q = 0; q < ps.nfl; ++q) {  // e-site flips (the paper's injection site)
      if (ps.fl[q].vec != V_E) continue;
      const long long g = ps.fl[q].g;
      const int j = (int)(g / nlon), i = (int)(g - (long long)j * nlon);
      T* v = sm + (j - rt.h0) * stride + sk(i);
      *v = flip_bits(*v, ps.fl[q].bit);
    }
  }
  if (sd.nlosses) {
    __syncthreads();  // thread 0's single flips are plain read-modify-writes
    apply_losses(sd, c.t, rt.h0, rt.h1, sm, stride);
  }
  __syncthreads();
}
// (3) L(e) on the own rows from the staged e rows (with halo rows), the dots
// and the tile's partial sums (write_e: also e itself and the norm an).
template <typename T, int KB>
__device__ __forceinline__ void step_stencil(const SolveDev<T>& sd, const Ctx<T>& c, const RowTile& rt, const T* sm,
                                             PhaseSmem& ps, double* part_out, const Acc<T>* an, bool write_e) {
  constexpr int W = V16<T>::W;
  constexpr bool kMixed = sizeof(T) == 4;
  const int nlon = sd.nlon, nlat = sd.nlat, stride = row_stride(nlon);
  Acc<T> ad[KB];
  Acc<T> ah, aq;  // mixed: <r', L(e)>, <L(e), L(e)>
  ah.mode(sd.oracle_order), aq.mode(sd.oracle_order);
#pragma unroll
  for (int l = 0; l < KB; ++l) ad[l].mode(sd.oracle_order);
  if (nlon % W == 0) {
    const int nvr = nlon / W, total = (rt.j1 - rt.j0) * nvr;
    for (int idx = threadIdx.x; idx < total; idx += kThreads) {
      const RowVec v = row_vec(idx, nvr, rt.j0, nlon, W);
      V16<T> rn;
      if constexpr (kMixed) rn = ldv(c.rW + v.g);  // r' of this step (written above)
      const bool hasN = v.j < nlat - 1, hasS = v.j > 0;
      const V16<T> tx = ldv_nc(sd.Tx + v.g);
      const T txw0 = __ldg(sd.Tx + (long long)v.j * nlon + (v.i == 0 ? nlon - 1 : v.i - 1));
      V16<T> ty, tys;
      if (hasN) ty = ldv_nc(sd.Ty + v.g);
      if (hasS) tys = ldv_nc(sd.Ty + v.g - nlon);
      const T muA = __ldg(sd.muA + v.j);
      V16<T> lpl[KB];
#pragma unroll
      for (int l = 0; l < KB; ++l)
        if (l <= c.nu) lpl[l] = ldv(c.lp[l] + v.g);
      const T* row = sm + (v.j - rt.h0) * stride;
      V16<T> ev, le;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const int i = v.i + w;
        const int ie = (i + 1 == nlon) ? 0 : i + 1;
        const int iw = (i == 0) ? nlon - 1 : i - 1;
        const T x = row[sk(i)];
        ev.v[w] = x;
        le.v[w] = stencil_op<T>(sd.oracle_order, x, row[sk(ie)], row[sk(iw)], hasN ? row[stride + sk(i)] : T(0),
                                hasS ? row[-stride + sk(i)] : T(0), tx.v[w], w == 0 ? txw0 : tx.v[w - 1],
                                hasN ? ty.v[w] : T(0), hasS ? tys.v[w] : T(0), muA, hasN, hasS);
      }
      if (write_e) stv(c.eW + v.g, ev);
      stv(c.LeW + v.g, le);
#pragma unroll
      for (int l = 0; l < KB; ++l)
        if (l <= c.nu) {
#pragma unroll
          for (int w = 0; w < W; ++w) ad[l].add(le.v[w], lpl[l].v[w]);
        }
      if constexpr (kMixed) {
#pragma unroll
        for (int w = 0; w < W; ++w) {
          ah.add(rn.v[w], le.v[w]);
          aq.add(le.v[w], le.v[w]);
        }
      }
    }
  } else {
    for (int j = rt.j0; j < rt.j1; ++j) {
      const long long base = (long long)j * nlon;
      const T* row = sm + (j - rt.h0) * stride;
      for (int i = threadIdx.x; i < nlon; i += kThreads) {
        const long long g = base + i;
        const T le = stencil_smem(sd, sm, stride, rt.h0, j, i);
        if (write_e) c.eW[g] = row[sk(i)];
        c.LeW[g] = le;
#pragma unroll
        for (int l = 0; l < KB; ++l)
          if (l <= c.nu) ad[l].add(le, ldcg(c.lp[l] + g));
        if constexpr (kMixed) {
          ah.add(ldcg(c.rW + g), le);
          aq.add(le, le);
        }
      }
    }
  }
  sub_mark(ps, 2);
  if (write_e) cta_red_put(ps.cr, 0, an->warp_sum());
#pragma unroll
  for (int l = 0; l < KB; ++l)
    if (l <= c.nu) cta_red_put(ps.cr, 1 + l, ad[l].warp_sum());
  if constexpr (kMixed) {
    cta_red_put(ps.cr, 2 + c.nu, ah.warp_sum());
    cta_red_put(ps.cr, 3 + c.nu, aq.warp_sum());
    cta_red_finish<T>(ps.cr, 4 + c.nu, part_out, write_e ? 0 : 1);
  } else {
    cta_red_finish<T>(ps.cr, 2 + c.nu, part_out, write_e ? 0 : 1);
  }
}

template <typename T, int KB, bool FUSED, bool GL = false>
__device__ __noinline__ void phase_pa(const SolveDev<T>& sd, const Ctx<T>& c, int sidx, int tau, T* sm, PhaseSmem& ps,
                                      double* part_out) {
  const int nlon = sd.nlon, nlat = sd.nlat, stride = row_stride(nlon);
  const RowTile rt = row_tile(nlat, sd.nt, tau);
  T* cs = sm + sd.cs_off;
  // a CTA that keeps the same tile keeps its staged constants (single solves)
  if (!(ps.cs_solve == sidx && ps.cs_tile == tau)) stage_line_consts<T, GL>(sd, rt.h0, rt.h1, cs);
  if (threadIdx.x == 0)
    ps.nfl = collect_flips(sd, c.t, FUSED ? (kStateVecs | (1u << V_E)) : (1u << V_E), (long long)rt.h0 * nlon,
                           (long long)rt.h1 * nlon, ps.fl);
  Acc<T> an;
  an.mode(sd.oracle_order);
  step_axpy<T, KB, FUSED>(sd, c, rt, sm, ps, an);
  step_precond<T, false, GL>(sd, c, rt, sm, cs, ps);
  step_stencil<T, KB>(sd, c, rt, sm, ps, part_out, &an, true);
  if (threadIdx.x == 0) {
    ps.cs_solve = sidx;
    ps.cs_tile = tau;
  }
}

// The step phase in the kernel instance with split rounds (wide rows, where
// shared memory leaves a tile few rows and recomputed halo rows would
// multiply the work).  mode 0: as phase_pa (a solve in one-pass rounds);
// mode 1, the first pass: the tile's own rows up to e, e written out, the norm
// as partial sum 0; mode 2, the second pass after a grid barrier: e of the own
// and halo rows read back, L(e), the dots.  One function for the three, as the
// instance's register allocation fares best with few phase functions.
template <typename T, int KB, bool FUSED>
__device__ __noinline__ void phase_pa_any(const SolveDev<T>& sd, const Ctx<T>& c, int sidx, int tau, T* sm,
                                          PhaseSmem& ps, double* part_out, int mode) {
  const int nlon = sd.nlon, stride = row_stride(nlon);
  RowTile rt = row_tile(sd.nlat, sd.nt, tau);
  Acc<T> an;
  an.mode(sd.oracle_order);
  if (mode == 2) {
    stage_rows(c.eW, rt.h0, rt.h1, nlon, sm, stride);
    if (sd.cs_clobber && threadIdx.x == 0) ps.cs_solve = -1;  // the rows overwrote staged constants
    __syncthreads();
  } else {
    if (mode == 1) {  // own rows only
      rt.h0 = rt.j0;
      rt.h1 = rt.j1;
    }
    T* cs = sm + sd.cs_off;
    if (!(ps.cs_solve == sidx && ps.cs_tile == tau)) stage_line_consts(sd, rt.h0, rt.h1, cs);
    if (threadIdx.x == 0)
      ps.nfl = collect_flips(sd, c.t, FUSED ? (kStateVecs | (1u << V_E)) : (1u << V_E), (long long)rt.h0 * nlon,
                             (long long)rt.h1 * nlon, ps.fl);
    step_axpy<T, KB, FUSED>(sd, c, rt, sm, ps, an);
    step_precond<T, true>(sd, c, rt, sm, cs, ps, mode == 1);
    if (threadIdx.x == 0) {
      ps.cs_solve = sidx;
      ps.cs_tile = tau;
    }
    if (mode == 1) {
      store_rows(c.eW, rt.h0, rt.h1, nlon, sm, stride);
      cta_red_put(ps.cr, 0, an.warp_sum());
      cta_red_finish<T>(ps.cr, 1, part_out);
      return;
    }
  }
  step_stencil<T, KB>(sd, c, rt, sm, ps, part_out, &an, mode == 0);
}

// PB: direction recurrences and the dots for the next beta.
template <typename T, int KB>
__device__ __noinline__ void phase_pb(const SolveDev<T>& sd, const Ctx<T>& c, int tau, PhaseSmem& ps, double* part_out) {
  constexpr int W = V16<T>::W;
  constexpr int U = 2;
  const long long e0 = elem_start(sd.N, sd.nt, tau), e1 = elem_start(sd.N, sd.nt, tau + 1);
  if (threadIdx.x == 0) ps.nfl = collect_flips(sd, c.t, kStateVecs, e0, e1, ps.fl);
  __syncthreads();
  const int nfl = ps.nfl;
  Acc<T> a0, a1;
  a0.mode(sd.oracle_order), a1.mode(sd.oracle_order);
  auto finish = [&](long long g, T pa, T la, T rv) {
    if (nfl) {
      pa = apply_flips(pa, g, V_P, nfl, ps.fl);
      la = apply_flips(la, g, V_AP, nfl, ps.fl);
      bool hitR = false;
      for (int q = 0; q < nfl; ++q) hitR = hitR || (ps.fl[q].g == g && ps.fl[q].vec == V_R);
      if (hitR) {
        rv = apply_flips(rv, g, V_R, nfl, ps.fl);
        c.rCw[g] = rv;
      }
      for (int q = 0; q < nfl; ++q)
        if (ps.fl[q].g == g && ps.fl[q].vec == V_X) c.phiCw[g] = flip_bits(ldcg(c.phiCw + g), ps.fl[q].bit);
    }
    c.pnew[g] = pa;
    c.lpnew[g] = la;
    a0.add(rv, la);
    a1.add(la, la);
  };
  const long long q0 = e0 / W, q1 = e1 / W;  // e0 is a multiple of 4
  for (long long b = q0 + threadIdx.x; b < q1; b += U * kThreads) {
    V16<T> pa[U], la[U], rv[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long q = b + (long long)u * kThreads;
      ok[u] = q < q1;
      if (ok[u]) {
        pa[u] = ldv(c.eR + q * W);
        la[u] = ldv(c.LeR + q * W);
        rv[u] = ldv(c.rCw + q * W);
      }
    }
#pragma unroll
    for (int l = 0; l < KB; ++l)
      if (l <= c.nu) {
        V16<T> pl[U], ll[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (ok[u]) {
            const long long q = b + (long long)u * kThreads;
            pl[u] = ldv(c.pp[l] + q * W);
            ll[u] = ldv(c.lp[l] + q * W);
          }
        const T al = c.alpha[l];
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (ok[u]) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
              pa[u].v[w] = tfma(al, pl[u].v[w], pa[u].v[w]);
              la[u].v[w] = tfma(al, ll[u].v[w], la[u].v[w]);
            }
          }
      }
#pragma unroll
    for (int u = 0; u < U; ++u)
      if (ok[u]) {
        const long long q = b + (long long)u * kThreads;
        if (nfl) {
#pragma unroll
          for (int w = 0; w < W; ++w) finish(q * W + w, pa[u].v[w], la[u].v[w], rv[u].v[w]);
        } else {
          stv(c.pnew + q * W, pa[u]);
          stv(c.lpnew + q * W, la[u]);
#pragma unroll
          for (int w = 0; w < W; ++w) {
            a0.add(rv[u].v[w], la[u].v[w]);
            a1.add(la[u].v[w], la[u].v[w]);
          }
        }
      }
  }
  for (long long g = q1 * W + threadIdx.x; g < e1; g += kThreads) {  // ragged tail
    T pa = ldcg(c.eR + g), la = ldcg(c.LeR + g);
    for (int l = 0; l < KB; ++l)
      if (l <= c.nu) {
        pa = tfma(c.alpha[l], ldcg(c.pp[l] + g), pa);
        la = tfma(c.alpha[l], ldcg(c.lp[l] + g), la);
      }
    finish(g, pa, la, ldcg(c.rCw + g));
  }
  cta_red_put(ps.cr, 0, a0.warp_sum());
  cta_red_put(ps.cr, 1, a1.warp_sum());
  cta_red_finish<T>(ps.cr, 2, part_out);
}

// RESTORE: [phi, r, p, L(p)]^0 <- [phi, r, p, L(p)]^* by copy (the backup
// itself is never the working set), then the flips of the next step.
template <typename T>
__device__ __noinline__ void phase_restore(const SolveDev<T>& sd, const Ctx<T>& c, int tau, PhaseSmem& ps, double* part_out) {
  const long long e0 = elem_start(sd.N, sd.nt, tau), e1 = elem_start(sd.N, sd.nt, tau + 1);
  if (threadIdx.x == 0) {
    ps.nfl = collect_flips(sd, c.t, kStateVecs, e0, e1, ps.fl);
    ps.npt = c.patched ? collect_flips(sd, c.patch_step, kStateVecs, e0, e1, ps.pt) : 0;
  }
  __syncthreads();
  const int nfl = ps.nfl, npt = ps.npt;
  Acc<T> a0, a1;
  a0.mode(sd.oracle_order), a1.mode(sd.oracle_order);
  for (long long g = e0 + threadIdx.x; g < e1; g += kThreads) {
    T ph = ldcg(c.phiS + g), rr = ldcg(c.rS + g), pp = ldcg(c.pS + g), ll = ldcg(c.lpS + g);
    if (npt) {
      ph = apply_patches(ph, g, V_X, npt, ps.pt, sd.patchval);
      rr = apply_patches(rr, g, V_R, npt, ps.pt, sd.patchval);
      pp = apply_patches(pp, g, V_P, npt, ps.pt, sd.patchval);
      ll = apply_patches(ll, g, V_AP, npt, ps.pt, sd.patchval);
    }
    if (nfl) {
      ph = apply_flips(ph, g, V_X, nfl, ps.fl);
      rr = apply_flips(rr, g, V_R, nfl, ps.fl);
      pp = apply_flips(pp, g, V_P, nfl, ps.fl);
      ll = apply_flips(ll, g, V_AP, nfl, ps.fl);
    }
    c.phiT[g] = ph;
    c.rT[g] = rr;
    c.pT[g] = pp;
    c.lpT[g] = ll;
    a0.add(rr, ll);
    a1.add(ll, ll);
  }
  cta_red_put(ps.cr, 0, a0.warp_sum());
  cta_red_put(ps.cr, 1, a1.warp_sum());
  cta_red_finish<T>(ps.cr, 2, part_out);
}

// The parts of INIT, inlined into the one-pass phase and the two passes of a
// split round.  (1) r0 into the staged rows [rt.h0, rt.h1), the own rows'
// x0, r0 written (with the step's x / r flips and their clean values kept).
template <typename T>
__device__ __forceinline__ void init_rows(const SolveDev<T>& sd, const Ctx<T>& c, const RowTile& rt, T* sm,
                                          PhaseSmem& ps, Acc<T>& an, Acc<T>& aR, AccF64& aR64, bool vec) {
  const int nlon = sd.nlon, nlat = sd.nlat, stride = row_stride(nlon);
  constexpr int W = V16<T>::W;
  const int nfl = ps.nfl;
  if (vec) {
    // r0 = -R_in (zero guess), x0 = 0; rin_R: r0 = -R (the caller's FP64 R,
    // 16-byte aligned here) and ||R||^2 in FP64
    const int nvr = nlon / W, total = (rt.h1 - rt.h0) * nvr;
    for (int idx = threadIdx.x; idx < total; idx += kThreads) {
      const RowVec v = row_vec(idx, nvr, rt.h0, nlon, W);
      V16<T> rin;
      if (c.rin_R) {
        constexpr int D2 = V16<double>::W;
#pragma unroll
        for (int h = 0; h < W; h += D2) {
          const V16<double> rr = ldv(sd.R + v.g + h);
#pragma unroll
          for (int w = 0; w < D2; ++w) {
            rin.v[h + w] = (T)rr.v[w];
            if (v.j >= rt.j0 && v.j < rt.j1) {
              if constexpr (sizeof(T) == 8)
                aR.add(rr.v[w], rr.v[w]);  // FP64 path: the compensated sum, as with x0 read
              else
                aR64.add(rr.v[w], rr.v[w]);
            }
          }
        }
      } else {
        rin = ldv(sd.Rin + v.g);
      }
      V16<T> rv, zv;
      T* row = sm + (v.j - rt.h0) * stride;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        // FP64 path from R: L(0) - R, whose zero entries are +0 (as with x0 read)
        rv.v[w] = (sizeof(T) == 8 && c.rin_R) ? T(0) - rin.v[w] : -rin.v[w];
        zv.v[w] = T(0);
        row[sk(v.i + w)] = rv.v[w];
      }
      if (v.j >= rt.j0 && v.j < rt.j1) {
#pragma unroll
        for (int w = 0; w < W; ++w) an.add(rv.v[w], rv.v[w]);
        stv(c.phiW + v.g, zv);
        stv(c.rW + v.g, rv);
      }
    }
  }
  for (int j = rt.h0; j < (vec ? rt.h0 : rt.h1); ++j) {
    const bool own = (j >= rt.j0 && j < rt.j1);
    T* row = sm + (j - rt.h0) * stride;
    const long long base = (long long)j * nlon;
    for (int i = threadIdx.x; i < nlon; i += kThreads) {
      const long long g = base + i;
      T rv, xv;
      if (c.rin_R) {
        const double Rg = ldcg(sd.R + g);
        rv = sizeof(T) == 8 ? T(0) - (T)Rg : -(T)Rg;  // FP64: L(0) - R; mixed: -(float)(R - 0)
        xv = T(0);
        if (own) {
          if constexpr (sizeof(T) == 8)
            aR.add(Rg, Rg);  // FP64 path: the compensated sum, as with x0 read
          else
            aR64.add(Rg, Rg);
        }
      } else if (c.zero_guess) {
        rv = -ldcg(sd.Rin + g);
        xv = T(0);
      } else {
        // FP64 path only (T = double): r0 = L(x0) - R
        const T Lx = (T)stencil_global<double>(sd.x0, sd.Tx64, sd.Ty64, sd.muA64, nlon, nlat, j, i, sd.oracle_order);
        rv = Lx - (T)ldcg(sd.R + g);
        xv = (T)ldcg(sd.x0 + g);
        if (own) aR.add((T)ldcg(sd.R + g), (T)ldcg(sd.R + g));
      }
      row[sk(i)] = rv;
      if (own) {
        an.add(rv, rv);
        if (nfl) {
          const T x2 = apply_flips(xv, g, V_X, nfl, ps.fl);
          const T r2 = apply_flips(rv, g, V_R, nfl, ps.fl);
          for (int q = 0; q < nfl; ++q) {
            if (ps.fl[q].g != g) continue;
            if (ps.fl[q].vec == V_X) sd.patchval[ps.fl[q].q] = (double)xv;
            if (ps.fl[q].vec == V_R) sd.patchval[ps.fl[q].q] = (double)rv;
          }
          xv = x2;
          rv = r2;
        }
        c.phiW[g] = xv;
        c.rW[g] = rv;
      }
    }
  }
}
// (2) L(p0) on the own rows from the staged p0 rows, the p / Ap flips, p0 and
// L(p0) written, the dots and the tile's partial sums (full: also ||r0||^2
// and ||R||^2).
template <typename T>
__device__ __forceinline__ void init_stencil(const SolveDev<T>& sd, const Ctx<T>& c, const RowTile& rt, const T* sm,
                                             PhaseSmem& ps, Acc<T>& a0, Acc<T>& a1, bool vec) {
  const int nlon = sd.nlon, nlat = sd.nlat, stride = row_stride(nlon);
  constexpr int W = V16<T>::W;
  const int nfl = ps.nfl;
  if (vec) {
    // p0 = P^-1 r0 (in the rows), L(p0) and the first dots, 16-byte accesses
    const int nvr = nlon / W, total = (rt.j1 - rt.j0) * nvr;
    for (int idx = threadIdx.x; idx < total; idx += kThreads) {
      const RowVec v = row_vec(idx, nvr, rt.j0, nlon, W);
      const bool hasN = v.j < nlat - 1, hasS = v.j > 0;
      const V16<T> tx = ldv_nc(sd.Tx + v.g);
      const T txw0 = __ldg(sd.Tx + (long long)v.j * nlon + (v.i == 0 ? nlon - 1 : v.i - 1));
      V16<T> ty, tys;
      if (hasN) ty = ldv_nc(sd.Ty + v.g);
      if (hasS) tys = ldv_nc(sd.Ty + v.g - nlon);
      const T muA = __ldg(sd.muA + v.j);
      const V16<T> rr = ldv(c.rW + v.g);
      const T* row = sm + (v.j - rt.h0) * stride;
      V16<T> pv, lv;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const int i = v.i + w;
        const int ie = (i + 1 == nlon) ? 0 : i + 1;
        const int iw = (i == 0) ? nlon - 1 : i - 1;
        const T x = row[sk(i)];
        pv.v[w] = x;
        lv.v[w] = stencil_op<T>(sd.oracle_order, x, row[sk(ie)], row[sk(iw)], hasN ? row[stride + sk(i)] : T(0),
                                hasS ? row[-stride + sk(i)] : T(0), tx.v[w], w == 0 ? txw0 : tx.v[w - 1],
                                hasN ? ty.v[w] : T(0), hasS ? tys.v[w] : T(0), muA, hasN, hasS);
        a0.add(rr.v[w], lv.v[w]);
        a1.add(lv.v[w], lv.v[w]);
      }
      stv(c.pnew + v.g, pv);
      stv(c.lpnew + v.g, lv);
    }
  }
  for (int j = rt.j0; j < (vec ? rt.j0 : rt.j1); ++j) {
    const long long base = (long long)j * nlon;
    const T* row = sm + (j - rt.h0) * stride;
    for (int i = threadIdx.x; i < nlon; i += kThreads) {
      const long long g = base + i;
      T lp = stencil_smem(sd, sm, stride, rt.h0, j, i);
      T pv = row[sk(i)];
      const T rv = ldcg(c.rW + g);
      if (nfl) {
        const T p2 = apply_flips(pv, g, V_P, nfl, ps.fl);
        const T l2 = apply_flips(lp, g, V_AP, nfl, ps.fl);
        for (int q = 0; q < nfl; ++q) {
          if (ps.fl[q].g != g) continue;
          if (ps.fl[q].vec == V_P) sd.patchval[ps.fl[q].q] = (double)pv;
          if (ps.fl[q].vec == V_AP) sd.patchval[ps.fl[q].q] = (double)lp;
        }
        pv = p2;
        lp = l2;
      }
      c.pnew[g] = pv;
      c.lpnew[g] = lp;
      a0.add(rv, lp);
      a1.add(lp, lp);
    }
  }
}
// The partial sums of INIT (full: also ||r0||^2 and ||R||^2).
template <typename T>
__device__ __forceinline__ void init_partials(PhaseSmem& ps, double* part_out, const Acc<T>* an, const Acc<T>* aR,
                                              const Acc<T>& a0, const Acc<T>& a1, bool full, const AccF64* aR64 = nullptr) {
  if (full) {
    cta_red_put(ps.cr, 0, an->warp_sum());
    cta_red_put(ps.cr, 1, aR64 ? aR64->warp_sum() : aR->warp_sum());
  }
  cta_red_put(ps.cr, 2, a0.warp_sum());
  cta_red_put(ps.cr, 3, a1.warp_sum());
  cta_red_finish<T>(ps.cr, 4, part_out, full ? 0 : 2);
}

// INIT: r0 = L(phi0) - R (FP64 path, phi0 = x0) or r0 = -R_in (mixed inner
// solve, phi0 = 0); p0 = P^-1(r0); L(p0); ||r0||^2, ||R||^2 and the first
// beta dots.  The x/r/p/Ap flips of the first step are applied to the working
// vectors, and their clean values kept so that the backup stays clean.
template <typename T, bool GL = false>
__device__ __noinline__ void phase_init(const SolveDev<T>& sd, const Ctx<T>& c, int sidx, int tau, T* sm, PhaseSmem& ps,
                           double* part_out) {
  const int nlon = sd.nlon, nlat = sd.nlat, stride = row_stride(nlon);
  const RowTile rt = row_tile(nlat, sd.nt, tau);
  if (threadIdx.x == 0)
    ps.nfl = collect_flips(sd, c.t, kStateVecs, (long long)rt.j0 * nlon, (long long)rt.j1 * nlon, ps.fl);
  T* cs = sm + sd.cs_off;
  if (!(ps.cs_solve == sidx && ps.cs_tile == tau)) stage_line_consts<T, GL>(sd, rt.h0, rt.h1, cs);
  __syncthreads();
  Acc<T> an, aR;
  an.mode(sd.oracle_order), aR.mode(sd.oracle_order);
  AccF64 aR64;
  constexpr int W = V16<T>::W;
  // the common case, 16-byte accesses (the caller's R must be aligned for them)
  const bool vec = c.zero_guess && ps.nfl == 0 && nlon % W == 0 &&
                   (!c.rin_R || (reinterpret_cast<unsigned long long>(sd.R) & 15ull) == 0ull);
  init_rows<T>(sd, c, rt, sm, ps, an, aR, aR64, vec);
  cp_async_wait_all();
  __syncthreads();
  precond_tile<T, false, GL>(sd, rt.h0, rt.h1 - rt.h0, sm, stride, cs);
  __syncthreads();
  Acc<T> a0, a1;
  a0.mode(sd.oracle_order), a1.mode(sd.oracle_order);
  init_stencil<T>(sd, c, rt, sm, ps, a0, a1, vec);
  init_partials<T>(ps, part_out, &an, &aR, a0, a1, true, c.rin_R && sizeof(T) == 4 ? &aR64 : nullptr);
  if (threadIdx.x == 0) {
    ps.cs_solve = sidx;
    ps.cs_tile = tau;
  }
}

// INIT in the kernel instance with split rounds.  mode 0: as phase_init;
// mode 1: r0 and p0 = P^-1(r0) of the own rows, p0 (unflipped) into the
// scratch vector e[0], the two norms; mode 2: p0 with its halo rows read back
// from e[0], L(p0), flips, dots.  Modes 1 and 2 walk the tile in sub-bands of
// at most sd.sub_h rows (the tall bands of streamed solves do not fit in
// shared memory at once); the sums run on over the sub-bands.
template <typename T>
__device__ __noinline__ void phase_init_any(const SolveDev<T>& sd, const Ctx<T>& c, int sidx, int tau, T* sm,
                                            PhaseSmem& ps, double* part_out, int mode) {
  const int nlon = sd.nlon, stride = row_stride(nlon);
  const RowTile rt = row_tile(sd.nlat, sd.nt, tau);
  if (threadIdx.x == 0)
    ps.nfl = collect_flips(sd, c.t, kStateVecs, (long long)rt.j0 * nlon, (long long)rt.j1 * nlon, ps.fl);
  Acc<T> an, aR, a0, a1;
  an.mode(sd.oracle_order), aR.mode(sd.oracle_order), a0.mode(sd.oracle_order), a1.mode(sd.oracle_order);
  AccF64 aR64;
  constexpr int W = V16<T>::W;
  const bool ralign = !c.rin_R || (reinterpret_cast<unsigned long long>(sd.R) & 15ull) == 0ull;
  const int sub = (mode == 0 || sd.sub_h <= 0) ? rt.j1 - rt.j0 : sd.sub_h;
  const bool one = sub >= rt.j1 - rt.j0;  // the whole tile at once
  for (int a = rt.j0; a < rt.j1; a += sub) {
    RowTile st;
    st.j0 = a;
    st.j1 = min(a + sub, rt.j1);
    st.h0 = st.j0 > 0 ? st.j0 - 1 : 0;
    st.h1 = st.j1 < sd.nlat ? st.j1 + 1 : sd.nlat;
    if (mode == 2) {
      if (!one) __syncthreads();  // the previous sub-band's rows are read
      stage_rows(sd.e[0], st.h0, st.h1, nlon, sm, stride);
      if (sd.cs_clobber && threadIdx.x == 0) ps.cs_solve = -1;
      __syncthreads();
    } else {
      if (mode == 1) {
        st.h0 = st.j0;
        st.h1 = st.j1;
      }
      T* cs = sm + sd.cs_off;
      if (!one) {
        __syncthreads();
        if (threadIdx.x == 0) ps.cs_solve = -1;
      }
      if (!(one && ps.cs_solve == sidx && ps.cs_tile == tau)) stage_line_consts(sd, st.h0, st.h1, cs);
      __syncthreads();
      const bool vec = c.zero_guess && ps.nfl == 0 && nlon % W == 0 && ralign;
      init_rows<T>(sd, c, st, sm, ps, an, aR, aR64, vec);
      cp_async_wait_all();
      __syncthreads();
      precond_tile<T, true>(sd, st.h0, st.h1 - st.h0, sm, stride, cs, mode == 1);
      __syncthreads();
      if (threadIdx.x == 0) {
        ps.cs_solve = one ? sidx : -1;
        ps.cs_tile = tau;
      }
      if (mode == 1) {
        store_rows(sd.e[0], st.h0, st.h1, nlon, sm, stride);
        continue;
      }
    }
    const bool vec = c.zero_guess && ps.nfl == 0 && nlon % W == 0;
    init_stencil<T>(sd, c, st, sm, ps, a0, a1, vec);
  }
  if (mode == 1) {
    cta_red_put(ps.cr, 0, an.warp_sum());
    cta_red_put(ps.cr, 1, c.rin_R && sizeof(T) == 4 ? aR64.warp_sum() : aR.warp_sum());
    cta_red_finish<T>(ps.cr, 2, part_out);
    return;
  }
  init_partials<T>(ps, part_out, &an, &aR, a0, a1, mode == 0, c.rin_R && sizeof(T) == 4 ? &aR64 : nullptr);
}

// OUT (mixed): x' = x + d in FP64, r_out = R - L64(x'), ||r_out||^2 (and
// ||R||^2 the first time), inner right-hand side R_in = (float) r_out.  The
// tile is walked in sub-bands of at most sd.sub_h rows (each staged with its
// halo rows) when it is taller than shared memory holds.
template <typename T>
__device__ __noinline__ void phase_out(const SolveDev<T>& sd, const Ctx<T>& c, int tau, double* smd, PhaseSmem& ps,
                          double* part_out) {
  const int nlon = sd.nlon, nlat = sd.nlat, stride = row_stride(nlon);
  const RowTile rtile = row_tile(nlat, sd.nt, tau);
  if (threadIdx.x == 0) ps.cs_solve = -1;  // its FP64 rows overwrite the staged constants
  AccF64 so, sR;
  const int sub = sd.sub_h > 0 ? sd.sub_h : rtile.j1 - rtile.j0;
  for (int a = rtile.j0; a < rtile.j1; a += sub) {
    RowTile rt;
    rt.j0 = a;
    rt.j1 = min(a + sub, rtile.j1);
    rt.h0 = rt.j0 > 0 ? rt.j0 - 1 : 0;
    rt.h1 = rt.j1 < nlat ? rt.j1 + 1 : nlat;
    if (a > rtile.j0) __syncthreads();  // the previous sub-band's rows are read
    int nz = 0;
    {
      // x' = x + d over the sub-band and its halo rows, as one flat loop so
      // that each thread keeps several loads in flight
      const int nrows = rt.h1 - rt.h0, total = nrows * nlon;
      constexpr int U = 4;
      for (int b = threadIdx.x; b < total; b += U * kThreads) {
        double xv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = b + u * kThreads;
          if (idx < total) {
            const long long g = (long long)rt.h0 * nlon + idx;
            xv[u] = c.xsrc ? ldcg(c.xsrc + g) : 0.0;  // x = 0 before a zero-guess solve's first OUT
            if (c.d) xv[u] = xv[u] + (double)ldcg(c.d + g);
          }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int idx = b + u * kThreads;
          if (idx < total) {
            const int jr = idx / nlon, i = idx - jr * nlon;
            smd[jr * stride + sk(i)] = xv[u];
            nz |= xv[u] != 0.0;
            const int j = rt.h0 + jr;
            if (j >= rt.j0 && j < rt.j1) c.xdst[(long long)rt.h0 * nlon + idx] = xv[u];
          }
        }
      }
    }
    // a sub-band whose x' (halo included) is all zero, as at the start of a
    // solve from a zero guess, has L64(x') = 0: skip the FP64 stencil
    const bool zero = !__syncthreads_or(nz);
    for (int j = rt.j0; j < rt.j1; ++j) {
      const long long base = (long long)j * nlon;
      const double* row = smd + (j - rt.h0) * stride;
      const bool hasN = j < nlat - 1, hasS = j > 0;
      if (zero) {
        for (int i = threadIdx.x; i < nlon; i += kThreads) {
          const long long g = base + i;
          const double Rv = ldcg(sd.R + g);
          const double ro = Rv - 0.0;
          sd.Rin[g] = (T)ro;
          so.add(ro, ro);
          if (c.first) sR.add(Rv, Rv);
        }
        continue;
      }
      for (int i = threadIdx.x; i < nlon; i += kThreads) {
        const long long g = base + i;
        const int ie = (i + 1 == nlon) ? 0 : i + 1;
        const int iw = (i == 0) ? nlon - 1 : i - 1;
        const double v = row[sk(i)];
        const double Lx = stencil5_fma(v, row[sk(ie)], row[sk(iw)], hasN ? row[stride + sk(i)] : 0.0,
                                       hasS ? row[-stride + sk(i)] : 0.0, __ldg(sd.Tx64 + g),
                                       __ldg(sd.Tx64 + base + iw), hasN ? __ldg(sd.Ty64 + g) : 0.0,
                                       hasS ? __ldg(sd.Ty64 + g - nlon) : 0.0, __ldg(sd.muA64 + j), hasN, hasS);
        const double Rv = ldcg(sd.R + g);
        const double ro = Rv - Lx;
        sd.Rin[g] = (T)ro;
        so.add(ro, ro);
        if (c.first) sR.add(Rv, Rv);
      }
    }
  }
  cta_red_put(ps.cr, 0, so.warp_sum());
  cta_red_put(ps.cr, 1, sR.warp_sum());
  cta_red_finish<T>(ps.cr, 2, part_out);
}

// FIN: write the solution to the caller's x and (FP64 path) the true
// residual ||L(x) - R||^2.
template <typename T>
__device__ __noinline__ void phase_fin(const SolveDev<T>& sd, const Ctx<T>& c, int tau, PhaseSmem& ps, double* part_out) {
  const int nlon = sd.nlon, nlat = sd.nlat;
  const RowTile rt = row_tile(nlat, sd.nt, tau);
  Acc<double> acc;
  acc.mode(sd.oracle_order);
  if (sd.mixed) {
    // the tile's rows are contiguous: a copy, four loads in flight per thread
    const double* xs = c.xsrc;
    const long long g0 = (long long)rt.j0 * nlon, g1 = (long long)rt.j1 * nlon;
    constexpr int U = 4;
    for (long long b = g0 + threadIdx.x; b < g1; b += U * kThreads) {
      double v[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long g = b + (long long)u * kThreads;
        if (g < g1) v[u] = xs ? ldcg(xs + g) : 0.0;  // no x buffer yet: x = 0
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const long long g = b + (long long)u * kThreads;
        if (g < g1) sd.xout[g] = v[u];
      }
    }
  } else {
    if (threadIdx.x == 0)
      ps.npt = c.patched ? collect_flips(sd, c.patch_step, 1u << V_X, 0, sd.N, ps.pt) : 0;
    __syncthreads();
    const int npt = ps.npt;
    const T* src = c.finsrc;
    for (int j = rt.j0; j < rt.j1; ++j) {
      const long long base = (long long)j * nlon;
      const bool hasN = j < nlat - 1, hasS = j > 0;
      for (int i = threadIdx.x; i < nlon; i += kThreads) {
        const long long g = base + i;
        const int ie = (i + 1 == nlon) ? 0 : i + 1;
        const int iw = (i == 0) ? nlon - 1 : i - 1;
        auto val = [&](long long q) -> double {
          if (c.finzero) return 0.0;
          double v = (double)ldcg(src + q);
          if (npt) v = (double)apply_patches((T)v, q, V_X, npt, ps.pt, sd.patchval);
          return v;
        };
        const double v = val(g);
        const double Lx = stencil_op<double>(sd.oracle_order, v, val(base + ie), val(base + iw),
                                             hasN ? val(g + nlon) : 0.0, hasS ? val(g - nlon) : 0.0, __ldg(sd.Tx64 + g),
                                             __ldg(sd.Tx64 + base + iw), hasN ? __ldg(sd.Ty64 + g) : 0.0,
                                             hasS ? __ldg(sd.Ty64 + g - nlon) : 0.0, __ldg(sd.muA64 + j), hasN, hasS);
        const double res = Lx - ldcg(sd.R + g);
        sd.xout[g] = v;
        acc.add(res, res);
      }
    }
  }
  cta_red_put(ps.cr, 0, acc.warp_sum());
  cta_red_finish<T>(ps.cr, 1, part_out);
}

}  // namespace ftgcr
#include "ftgcr_stream.cuh"
namespace ftgcr {

// ------------------------------------------------------------ the kernel
// Block-wide copies of the per-solve records.  Records written during the
// kernel by other CTAs are read through L2 (ld.global.cg).
template <typename S>
__device__ __forceinline__ void cta_load_cg(S* dst, const S* src) {
  static_assert(sizeof(S) % 8 == 0, "record size");
  const long long* s = reinterpret_cast<const long long*>(src);
  long long* d = reinterpret_cast<long long*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(S) / 8); i += blockDim.x) d[i] = __ldcg(s + i);
}
template <typename S>
__device__ __forceinline__ void cta_zero(S* dst) {
  static_assert(sizeof(S) % 8 == 0, "record size");
  long long* d = reinterpret_cast<long long*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(S) / 8); i += blockDim.x) d[i] = 0;
}
template <typename S>
__device__ __forceinline__ void cta_store(S* dst, const S* src) {
  static_assert(sizeof(S) % 8 == 0, "record size");
  const long long* s = reinterpret_cast<const long long*>(src);
  long long* d = reinterpret_cast<long long*>(dst);
  for (int i = threadIdx.x; i < (int)(sizeof(S) / 8); i += blockDim.x) d[i] = s[i];
}

template <typename T>
struct KernelSmem {
  SolveDev<T> sd;
  SolveState S;
  SolveState N;
  Ctx<T> c;
  PhaseSmem ps;
  double red[kNPart];
  double qd[32];
  int prefix[kMaxBatch + 1];
  int bail;
};

// Loop state of a CTA (the same in every thread).
struct LoopState {
  int cur_sd = -1;            // solve whose descriptor sits in ks.sd
  int last_s = -1;            // solve whose transition ks.N holds, and its round
  long long last_round = -2;
  int cur = -1;               // solve whose context ks.c holds this round
  int spec_s = -1;            // solve whose partial sums ks.red holds already (speculative)
  bool red_ready = false;
};

// Entering solve s in a round: its descriptor, its state record and every
// partial sum the pending phase may have left, this round's transition into
// ks.N and ks.c.  A CTA that ran this solve's transition in the previous
// round holds the record already (every CTA computes the same transition
// from the same inputs).
template <typename T>
__device__ __forceinline__ void enter_solve(SolveDev<T>* const* solves, KernelSmem<T>& ks, LoopState& ls, int s,
                                            int par, long long round) {
  if (s != ls.cur_sd) {
    cta_load_cg(&ks.sd, solves[s]);
    __syncthreads();
    ls.cur_sd = s;
  }
  if (s == ls.last_s && round == ls.last_round + 1)
    cta_store(&ks.S, &ks.N);
  else
    cta_load_cg(&ks.S, ks.sd.st + par);
  if (!(ls.red_ready && s == ls.spec_s))
    reduce_partials<T>(ks.sd.part + (long long)(par ^ 1) * ks.sd.nt * kPartStride, ks.sd.nt, part_values(ks.sd),
                       ks.red);
  ls.red_ready = false;
  __syncthreads();
  precompute_divisions(ks.S, ks.red, ks.qd, ks.sd.mixed);
  cta_store(&ks.N, &ks.S);
  cta_zero(&ks.c);
  __syncthreads();
  if (threadIdx.x == 0) transition(ks.sd, ks.S, ks.red, ks.qd, ks.N, ks.c);
  __syncthreads();
  fill_directions(ks.sd, ks.S, ks.N, ks.qd, ks.c);
  __syncthreads();
  ls.cur = s;
  ls.last_s = s;
  ls.last_round = round;
}

// The phase of tile tau of the solve in ks.  pass 0: a one-pass round, or the
// first pass of a split round; pass 1: the second pass of a split round (the
// step phases of split solves only).
template <typename T, int KB, int WIDE>
__device__ __forceinline__ void run_phase(KernelSmem<T>& ks, int pass, int s, int tau, T* sm, double* part_out,
                                          int* err) {
  const int kind = ks.c.kind;
  if constexpr (WIDE != 0 && sizeof(T) == 4) {
    const int mode = ks.sd.split ? 1 + pass : 0;
    if (pass == 1 && mode == 0) return;
    if constexpr (WIDE == 2) {
      // streamed solves: the step rounds stream rows; the other rounds run as
      // split rounds over sub-bands
      if (ks.sd.split == 2 && kind == K_PA) {
        phase_stream<KB, false>(ks.sd, ks.c, tau, sm, ks.ps, part_out, pass, err);
        return;
      }
      if (ks.sd.split == 2 && kind == K_PF) {
        phase_stream<KB, true>(ks.sd, ks.c, tau, sm, ks.ps, part_out, pass, err);
        return;
      }
    }
    switch (kind) {
      case K_INIT: phase_init_any<T>(ks.sd, ks.c, s, tau, sm, ks.ps, part_out, mode); return;
      case K_PA: phase_pa_any<T, KB, false>(ks.sd, ks.c, s, tau, sm, ks.ps, part_out, mode); return;
      case K_PF: phase_pa_any<T, KB, true>(ks.sd, ks.c, s, tau, sm, ks.ps, part_out, mode); return;
      default:
        if (pass == 1) return;
        break;
    }
  } else {
    switch (kind) {
      case K_INIT: phase_init<T, WIDE != 0>(ks.sd, ks.c, s, tau, sm, ks.ps, part_out); return;
      case K_PA: phase_pa<T, KB, false, WIDE != 0>(ks.sd, ks.c, s, tau, sm, ks.ps, part_out); return;
      case K_PF:
        if constexpr (sizeof(T) == 4) phase_pa<T, KB, true>(ks.sd, ks.c, s, tau, sm, ks.ps, part_out);
        return;
      default: break;
    }
  }
  switch (kind) {
    case K_PB: phase_pb<T, KB>(ks.sd, ks.c, tau, ks.ps, part_out); break;
    case K_RESTORE: phase_restore(ks.sd, ks.c, tau, ks.ps, part_out); break;
    case K_OUT: phase_out(ks.sd, ks.c, tau, reinterpret_cast<double*>(sm), ks.ps, part_out); break;
    case K_FIN: phase_fin(ks.sd, ks.c, tau, ks.ps, part_out); break;
    default: break;
  }
}

// Persistent cooperative kernel: every round, every CTA takes its share of
// the tiles of all active solves, runs for each solve the state transition
// and the decided phase, and then meets the others at one grid barrier.
// WIDE 1: the instance for launches with wide-row solves.  Mixed path: solves
// with split rounds, whose every round takes a second pass over the tiles
// after a further barrier.  FP64 path: solves whose line solve reads its
// factors from global memory.  WIDE 2 (mixed path): that instance plus the
// streamed step rounds of HBM-resident solves.  The plain instance carries
// none of that code.
template <typename T, int KB, int WIDE>
__global__ void __launch_bounds__(kThreads, 1) k_ftgcr_persistent(BatchArgs<T> a) {
  constexpr bool SPLIT = WIDE != 0 && sizeof(T) == 4;  // split rounds: mixed path only
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ KernelSmem<T> ks;
  T* sm = reinterpret_cast<T*>(dsm);
  if constexpr (WIDE == 2 && sizeof(T) == 4) stream_init();
  const long long round0 = a.ctl->round0;
  const unsigned long long t_start = globaltimer();
  unsigned int nbar = 0;
  LoopState ls;
  if (threadIdx.x == 0) ks.ps.cs_solve = -1;
  int it = 0;
  for (; it < a.max_rounds; ++it) {
    // watchdog: a kernel that runs far longer than any solve raises the error
    // flag; every CTA leaves at its next barrier
    if (threadIdx.x == 0 && globaltimer() - t_start > kKernelTimeoutNs) atomicExch(&a.ctl->err, 2);
    const long long round = round0 + it;
    const int par = (int)(round & 1);
    if (threadIdx.x == 0 && a.diag) {
      a.diag[blockIdx.x * 4 + 0] = it;
      a.diag[blockIdx.x * 4 + 2] = 0;
    }
    // speculative: a CTA that ran a solve's transition last round will most
    // likely run the same solve first this round; warps 1.. reduce its
    // partial sums while warp 0 forms the tile prefix
    const int spec_s = (ls.cur_sd >= 0 && ls.last_s == ls.cur_sd && ls.last_round == round - 1) ? ls.cur_sd : -1;
    ls.spec_s = spec_s;
    ls.red_ready = spec_s >= 0;
    ls.cur = -1;
    if (spec_s >= 0)
      reduce_partials<T>(ks.sd.part + (long long)(par ^ 1) * ks.sd.nt * kPartStride, ks.sd.nt, part_values(ks.sd),
                         ks.red, 1);
    // tile prefix over active solves (identical in every CTA): warp 0 scans
    // 32 solves at a time
    if (threadIdx.x < 32) {
      const int lane = threadIdx.x;
      int acc = 0;
      for (int s0 = 0; s0 < a.n; s0 += 32) {
        const int s = s0 + lane;
        int v = 0;
        if (s < a.n) {
          const int act = __ldcg(a.active + par * a.n + s);
          v = act ? a.nt[s] : 0;
          if (!act && blockIdx.x == 0) a.active[(par ^ 1) * a.n + s] = 0;
        }
        int inc = v;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, inc, d);
          if (lane >= d) inc += y;
        }
        if (s < a.n) ks.prefix[s] = acc + inc - v;
        acc += __shfl_sync(0xffffffffu, inc, 31);
      }
      if (lane == 0) ks.prefix[a.n] = acc;
    }
    __syncthreads();
    const int total = ks.prefix[a.n];
    if (total == 0) break;
    unsigned long long tr0 = 0ull, tr1 = 0ull, tr2 = 0ull;
    int tr_kind = -1, tr_items = 0;
    if (a.trace && threadIdx.x == 0) tr0 = globaltimer();
    if (threadIdx.x == 0) {
      ks.ps.tracing = a.trace != nullptr;
      ks.ps.sub[0] = ks.ps.sub[1] = ks.ps.sub[2] = 0ull;
    }
    constexpr int npass = SPLIT ? 2 : 1;
    for (int pass = 0; pass < npass; ++pass) {
      if (pass == 1) {
        // second pass of split rounds: after every tile's e is written,
        // L(e) and the dots of the split solves' tiles
        ++nbar;
        if (!grid_barrier(&a.ctl->counter, nbar * gridDim.x, &a.ctl->err, &ks.bail)) return;
      }
      for (int item = blockIdx.x; item < total; item += gridDim.x) {
        int lo = 0, hi = a.n - 1;  // the last solve s with prefix[s] <= item
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (ks.prefix[mid] <= item) lo = mid; else hi = mid - 1;
        }
        const int s = lo;
        const int tau = item - ks.prefix[s];
        if (s != ls.cur) enter_solve<T>(a.solves, ks, ls, s, par, round);
        if (pass == 0) {
          if (a.trace && threadIdx.x == 0 && tr_items == 0) {
            tr1 = globaltimer();
            tr_kind = ks.c.kind;
          }
          ++tr_items;
          if (threadIdx.x == 0 && a.diag) {
            a.diag[blockIdx.x * 4 + 1] = ks.c.kind;
            a.diag[blockIdx.x * 4 + 2] = 1;
            a.diag[blockIdx.x * 4 + 3] = tr_items;
          }
        }
        run_phase<T, KB, WIDE>(ks, pass, s, tau, sm, ks.sd.part + ((long long)par * ks.sd.nt + tau) * kPartStride,
                               &a.ctl->err);
        __syncthreads();
        if (pass == 0 && tau == 0) {
          cta_store(ks.sd.st + (par ^ 1), &ks.N);
          if (!ks.N.active) cta_store(ks.sd.result, &ks.N);
          if (threadIdx.x == 0) a.active[(par ^ 1) * a.n + s] = ks.N.active;
          __syncthreads();
        }
      }
    }
    if (a.trace && threadIdx.x == 0) tr2 = globaltimer();
    if (threadIdx.x == 0 && a.diag) a.diag[blockIdx.x * 4 + 2] = 2;
    ++nbar;
    const bool ok = grid_barrier(&a.ctl->counter, nbar * gridDim.x, &a.ctl->err, &ks.bail);
    if (a.trace && threadIdx.x == 0 && it < a.trace_rounds) {
      TraceEnt e;
      e.t0 = tr0;
      e.t1 = tr1;
      e.t2 = tr2;
      e.t3 = globaltimer();
      e.s0 = ks.ps.sub[0];
      e.s1 = ks.ps.sub[1];
      e.s2 = ks.ps.sub[2];
      e.kind = tr_kind;
      e.items = tr_items;
      a.trace[(long long)it * gridDim.x + blockIdx.x] = e;
    }
    if (!ok) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->round_end = round0 + it;
}

}  // namespace ftgcr
