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
};

template <typename T>
struct BatchArgs {
  SolveDev<T>* const* solves;  // [n]
  const int* nt;               // [n] tiles per solve
  int* active;                 // [2][n]
  int n;
  LaunchCtl* ctl;
  int max_rounds;
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

// ------------------------------------------------------------ reductions
// Deterministic sum of value v over the nt tiles of the partials buffer, by
// warp 0; every CTA that works on the solve gets the identical result.
__device__ __forceinline__ void reduce_partials(const double* part, int nt, int nv, double* red) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    for (int v = 0; v < nv; ++v) {
      double s = 0.0;
      for (int tau = lane; tau < nt; tau += 32) s += __ldcg(part + (long long)tau * kNPart + v);
      s = warp_sum(s);
      if (lane == 0) red[v] = s;
    }
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

// Number of partial sums the phase `kind` leaves per tile.
__device__ __forceinline__ int part_count(int kind, int nu) {
  switch (kind) {
    case K_INIT: return 4;
    case K_PA: return 2 + nu;
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
__device__ void transition(const SolveDev<T>& sd, const SolveState& S, const double* red, SolveState& N, Ctx<T>& c) {
  N = S;
  c.kind = K_NONE;
  c.zero_guess = 0;
  c.xsrc_user = 0;
  c.finzero = 0;
  c.first = 0;
  c.patched = 0;
  c.nu = S.nu;
  c.t = S.step + 1;
  c.patch_step = S.step + 1;
  int dbuf = -1;       // OUT: phi buffer holding the inner solution
  int finbuf = -1;     // FIN: phi buffer holding the iterate to return
  bool to_out = false; // mixed: leave the inner solve
  bool to_fin = false;
  switch (S.pending) {
    case K_NONE:
      if (sd.mixed) {
        c.kind = K_OUT;
        c.xsrc_user = 1;
        c.first = 1;
      } else {
        c.kind = K_INIT;
      }
      break;
    case K_OUT: {
      const double nrm2_out = red[0];
      if (S.first_out) {
        N.nrm2_R = red[1];
        N.thr2 = sd.tol2 * N.nrm2_R;
        N.first_out = 0;
        N.nrm2_0 = nrm2_out;
      }
      N.xcur = S.xcur ^ 1;
      N.nrm2_out = nrm2_out;
      N.outer = S.outer + 1;
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
        N.beta = -red[2] / red[3];
        N.lpn2[0] = red[3];
        c.kind = K_PA;
      }
      break;
    }
    case K_PA: {
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
      } else if (!(nrm2 < S.nrm2_prev)) {  // fault test (Algorithm 1, red part)
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
        for (int l = 0; l < kMaxK; ++l)
          if (l <= S.nu) c.alpha[l] = (T)(-red[1 + l] / S.lpn2[l]);
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
        }
      }
      break;
    }
    case K_PB:
    case K_RESTORE:
      N.finj = S.finj + count_faults(sd, S.step + 1, kStateVecs);
      N.beta = -red[0] / red[1];
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
  if (c.kind == K_PA) {
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
    for (int l = 0; l < kMaxK; ++l)
      if (l <= N.nu) c.lp[l] = sd.Lp[N.slot[l]];
  } else if (c.kind == K_PB) {
    for (int l = 0; l < kMaxK; ++l)
      if (l <= S.nu) {
        c.pp[l] = sd.p[S.slot[l]];
        c.lp[l] = sd.Lp[S.slot[l]];
      }
    c.phiCw = sd.phi[N.phiC];
    c.rCw = sd.r[N.rC];
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
  } else if (c.kind == K_OUT) {
    c.xsrc = c.xsrc_user ? sd.x0 : sd.xbuf[S.xcur];
    c.xdst = sd.xbuf[S.xcur ^ 1];
  } else if (c.kind == K_FIN) {
    if (sd.mixed) c.xsrc = sd.xbuf[N.xcur];
  }
  N.pending = c.kind;
  if (c.kind == K_NONE) N.active = 0;
}

// ------------------------------------------------------------ phases
template <typename T>
struct PhaseSmem {
  FlipEnt fl[kMaxFaults];
  FlipEnt pt[kMaxFaults];
  int nfl, npt;
  double red[kWarps * kNPart];
};

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
  return stencil5<T>(v, row[sk(ie)], row[sk(iw)], vn, vs, __ldg(sd.Tx + g), __ldg(sd.Tx + (long long)j * nlon + iw),
                     hasN ? __ldg(sd.Ty + g) : T(0), hasS ? __ldg(sd.Ty + g - nlon) : T(0), __ldg(sd.muA + j), hasN,
                     hasS);
}

// Stencil on a global-memory field (initialisation / final residual).
template <typename V>
__device__ __forceinline__ V stencil_global(const V* x, const V* Tx, const V* Ty, const V* muA, int nlon, int nlat,
                                            int j, int i) {
  const int ie = (i + 1 == nlon) ? 0 : i + 1;
  const int iw = (i == 0) ? nlon - 1 : i - 1;
  const long long g = (long long)j * nlon + i;
  const bool hasN = j < nlat - 1, hasS = j > 0;
  const V v = ldcg(x + g);
  const V vn = hasN ? ldcg(x + g + nlon) : V(0);
  const V vs = hasS ? ldcg(x + g - nlon) : V(0);
  return stencil5<V>(v, ldcg(x + (long long)j * nlon + ie), ldcg(x + (long long)j * nlon + iw), vn, vs, __ldg(Tx + g),
                     __ldg(Tx + (long long)j * nlon + iw), hasN ? __ldg(Ty + g) : V(0), hasS ? __ldg(Ty + g - nlon) : V(0),
                     __ldg(muA + j), hasN, hasS);
}

// PA: axpy, norm, preconditioner, operator, orthogonalisation dots.
template <typename T>
__device__ void phase_pa(const SolveDev<T>& sd, const Ctx<T>& c, int tau, T* sm, PhaseSmem<T>& ps, double* part_out) {
  const int nlon = sd.nlon, stride = row_stride(nlon);
  const RowTile rt = row_tile(sd.nlat, sd.nt, tau);
  const int warp = threadIdx.x >> 5;
  const T beta = c.beta;
  Acc<T> an;
  for (int j = rt.h0; j < rt.h1; ++j) {
    const bool own = (j >= rt.j0 && j < rt.j1);
    T* row = sm + (j - rt.h0) * stride;
    const long long base = (long long)j * nlon;
    for (int i = threadIdx.x; i < nlon; i += kThreads) {
      const long long g = base + i;
      const T rv = tfma(beta, ldcg(c.lpnu + g), ldcg(c.rC + g));
      row[sk(i)] = rv;
      if (own) {
        c.rW[g] = rv;
        c.phiW[g] = tfma(beta, ldcg(c.pnu + g), ldcg(c.phiC + g));
        an.add(rv, rv);
      }
    }
  }
  if (threadIdx.x == 0)
    ps.nfl = collect_flips(sd, c.t, 1u << V_E, (long long)rt.h0 * nlon, (long long)rt.h1 * nlon, ps.fl);
  __syncthreads();
  for (int jr = warp; jr < rt.h1 - rt.h0; jr += kWarps) precond_row(sd, rt.h0 + jr, sm + jr * stride);
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < ps.nfl; ++q) {  // e-site flips (paper's injection site)
      const long long g = ps.fl[q].g;
      const int j = (int)(g / nlon), i = (int)(g - (long long)j * nlon);
      T* v = sm + (j - rt.h0) * stride + sk(i);
      *v = flip_bits(*v, ps.fl[q].bit);
    }
  }
  __syncthreads();
  Acc<T> ad[kMaxK];
  for (int j = rt.j0; j < rt.j1; ++j) {
    const long long base = (long long)j * nlon;
    const T* row = sm + (j - rt.h0) * stride;
    for (int i = threadIdx.x; i < nlon; i += kThreads) {
      const long long g = base + i;
      const T le = stencil_smem(sd, sm, stride, rt.h0, j, i);
      sd.e[g] = row[sk(i)];
      sd.Le[g] = le;
#pragma unroll
      for (int l = 0; l < kMaxK; ++l)
        if (l <= c.nu) ad[l].add(le, ldcg(c.lp[l] + g));
    }
  }
  // deterministic CTA reduction of 2 + nu values
  const int lane = threadIdx.x & 31;
  {
    double s = warp_sum(an.get());
    if (lane == 0) ps.red[warp * kNPart + 0] = s;
  }
#pragma unroll
  for (int l = 0; l < kMaxK; ++l)
    if (l <= c.nu) {
      double s = warp_sum(ad[l].get());
      if (lane == 0) ps.red[warp * kNPart + 1 + l] = s;
    }
  __syncthreads();
  if (threadIdx.x < 2 + c.nu) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += ps.red[w * kNPart + threadIdx.x];
    part_out[threadIdx.x] = s;
  }
}

// PB: direction recurrences and the dots for the next beta.
template <typename T>
__device__ void phase_pb(const SolveDev<T>& sd, const Ctx<T>& c, int tau, PhaseSmem<T>& ps, double* part_out) {
  const long long e0 = elem_start(sd.N, sd.nt, tau), e1 = elem_start(sd.N, sd.nt, tau + 1);
  if (threadIdx.x == 0) ps.nfl = collect_flips(sd, c.t, kStateVecs, e0, e1, ps.fl);
  __syncthreads();
  const int nfl = ps.nfl;
  Acc<T> a0, a1;
  for (long long g = e0 + threadIdx.x; g < e1; g += kThreads) {
    T pa = ldcg(sd.e + g), la = ldcg(sd.Le + g);
#pragma unroll
    for (int l = 0; l < kMaxK; ++l)
      if (l <= c.nu) {
        pa = tfma(c.alpha[l], ldcg(c.pp[l] + g), pa);
        la = tfma(c.alpha[l], ldcg(c.lp[l] + g), la);
      }
    T rv = ldcg(c.rCw + g);
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
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s0 = warp_sum(a0.get()), s1 = warp_sum(a1.get());
  if (lane == 0) {
    ps.red[warp * kNPart + 0] = s0;
    ps.red[warp * kNPart + 1] = s1;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += ps.red[w * kNPart + threadIdx.x];
    part_out[threadIdx.x] = s;
  }
}

// RESTORE: [phi, r, p, L(p)]^0 <- [phi, r, p, L(p)]^* by copy (the backup
// itself is never the working set), then the flips of the next step.
template <typename T>
__device__ void phase_restore(const SolveDev<T>& sd, const Ctx<T>& c, int tau, PhaseSmem<T>& ps, double* part_out) {
  const long long e0 = elem_start(sd.N, sd.nt, tau), e1 = elem_start(sd.N, sd.nt, tau + 1);
  if (threadIdx.x == 0) {
    ps.nfl = collect_flips(sd, c.t, kStateVecs, e0, e1, ps.fl);
    ps.npt = c.patched ? collect_flips(sd, c.patch_step, kStateVecs, e0, e1, ps.pt) : 0;
  }
  __syncthreads();
  const int nfl = ps.nfl, npt = ps.npt;
  Acc<T> a0, a1;
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
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double s0 = warp_sum(a0.get()), s1 = warp_sum(a1.get());
  if (lane == 0) {
    ps.red[warp * kNPart + 0] = s0;
    ps.red[warp * kNPart + 1] = s1;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += ps.red[w * kNPart + threadIdx.x];
    part_out[threadIdx.x] = s;
  }
}

// INIT: r0 = L(phi0) - R (FP64 path, phi0 = x0) or r0 = -R_in (mixed inner
// solve, phi0 = 0); p0 = P^-1(r0); L(p0); ||r0||^2, ||R||^2 and the first
// beta dots.  The x/r/p/Ap flips of the first step are applied to the working
// vectors, and their clean values kept so that the backup stays clean.
template <typename T>
__device__ void phase_init(const SolveDev<T>& sd, const Ctx<T>& c, int tau, T* sm, PhaseSmem<T>& ps,
                           double* part_out) {
  const int nlon = sd.nlon, nlat = sd.nlat, stride = row_stride(nlon);
  const RowTile rt = row_tile(nlat, sd.nt, tau);
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x == 0)
    ps.nfl = collect_flips(sd, c.t, kStateVecs, (long long)rt.j0 * nlon, (long long)rt.j1 * nlon, ps.fl);
  __syncthreads();
  const int nfl = ps.nfl;
  Acc<T> an, aR;
  for (int j = rt.h0; j < rt.h1; ++j) {
    const bool own = (j >= rt.j0 && j < rt.j1);
    T* row = sm + (j - rt.h0) * stride;
    const long long base = (long long)j * nlon;
    for (int i = threadIdx.x; i < nlon; i += kThreads) {
      const long long g = base + i;
      T rv, xv;
      if (c.zero_guess) {
        rv = -ldcg(sd.Rin + g);
        xv = T(0);
      } else {
        // FP64 path only (T = double): r0 = L(x0) - R
        const T Lx = (T)stencil_global<double>(sd.x0, sd.Tx64, sd.Ty64, sd.muA64, nlon, nlat, j, i);
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
  __syncthreads();
  for (int jr = warp; jr < rt.h1 - rt.h0; jr += kWarps) precond_row(sd, rt.h0 + jr, sm + jr * stride);
  __syncthreads();
  Acc<T> a0, a1;
  for (int j = rt.j0; j < rt.j1; ++j) {
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
  const int lane = threadIdx.x & 31;
  double v[4] = {an.get(), aR.get(), a0.get(), a1.get()};
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    double s = warp_sum(v[q]);
    if (lane == 0) ps.red[warp * kNPart + q] = s;
  }
  __syncthreads();
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += ps.red[w * kNPart + threadIdx.x];
    part_out[threadIdx.x] = s;
  }
}

// OUT (mixed): x' = x + d in FP64, r_out = R - L64(x'), ||r_out||^2 (and
// ||R||^2 the first time), inner right-hand side R_in = (float) r_out.
template <typename T>
__device__ void phase_out(const SolveDev<T>& sd, const Ctx<T>& c, int tau, double* smd, PhaseSmem<T>& ps,
                          double* part_out) {
  const int nlon = sd.nlon, nlat = sd.nlat, stride = row_stride(nlon);
  const RowTile rt = row_tile(nlat, sd.nt, tau);
  const int warp = threadIdx.x >> 5;
  for (int j = rt.h0; j < rt.h1; ++j) {
    const bool own = (j >= rt.j0 && j < rt.j1);
    double* row = smd + (j - rt.h0) * stride;
    const long long base = (long long)j * nlon;
    for (int i = threadIdx.x; i < nlon; i += kThreads) {
      const long long g = base + i;
      double xv = ldcg(c.xsrc + g);
      if (c.d) xv = xv + (double)ldcg(c.d + g);
      row[sk(i)] = xv;
      if (own) c.xdst[g] = xv;
    }
  }
  __syncthreads();
  double so = 0.0, sR = 0.0;
  for (int j = rt.j0; j < rt.j1; ++j) {
    const long long base = (long long)j * nlon;
    const double* row = smd + (j - rt.h0) * stride;
    const bool hasN = j < nlat - 1, hasS = j > 0;
    for (int i = threadIdx.x; i < nlon; i += kThreads) {
      const long long g = base + i;
      const int ie = (i + 1 == nlon) ? 0 : i + 1;
      const int iw = (i == 0) ? nlon - 1 : i - 1;
      const double v = row[sk(i)];
      const double Lx = stencil5<double>(v, row[sk(ie)], row[sk(iw)], hasN ? row[stride + sk(i)] : 0.0,
                                         hasS ? row[-stride + sk(i)] : 0.0, __ldg(sd.Tx64 + g),
                                         __ldg(sd.Tx64 + base + iw), hasN ? __ldg(sd.Ty64 + g) : 0.0,
                                         hasS ? __ldg(sd.Ty64 + g - nlon) : 0.0, __ldg(sd.muA64 + j), hasN, hasS);
      const double Rv = ldcg(sd.R + g);
      const double ro = Rv - Lx;
      sd.Rin[g] = (T)ro;
      so = fma(ro, ro, so);
      if (c.first) sR = fma(Rv, Rv, sR);
    }
  }
  const int lane = threadIdx.x & 31;
  double s0 = warp_sum(so), s1 = warp_sum(sR);
  if (lane == 0) {
    ps.red[warp * kNPart + 0] = s0;
    ps.red[warp * kNPart + 1] = s1;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    double s = 0.0;
    for (int w = 0; w < kWarps; ++w) s += ps.red[w * kNPart + threadIdx.x];
    part_out[threadIdx.x] = s;
  }
}

// FIN: write the solution to the caller's x and (FP64 path) the true
// residual ||L(x) - R||^2.
template <typename T>
__device__ void phase_fin(const SolveDev<T>& sd, const Ctx<T>& c, int tau, PhaseSmem<T>& ps, double* part_out) {
  const int nlon = sd.nlon, nlat = sd.nlat;
  const RowTile rt = row_tile(nlat, sd.nt, tau);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  double acc = 0.0;
  if (sd.mixed) {
    const double* xs = c.xsrc;
    for (long long g = (long long)rt.j0 * nlon + threadIdx.x; g < (long long)rt.j1 * nlon; g += kThreads)
      sd.xout[g] = ldcg(xs + g);
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
        const double Lx = stencil5<double>(v, val(base + ie), val(base + iw), hasN ? val(g + nlon) : 0.0,
                                           hasS ? val(g - nlon) : 0.0, __ldg(sd.Tx64 + g), __ldg(sd.Tx64 + base + iw),
                                           hasN ? __ldg(sd.Ty64 + g) : 0.0, hasS ? __ldg(sd.Ty64 + g - nlon) : 0.0,
                                           __ldg(sd.muA64 + j), hasN, hasS);
        const double res = Lx - ldcg(sd.R + g);
        sd.xout[g] = v;
        acc = fma(res, res, acc);
      }
    }
  }
  double s = warp_sum(acc);
  if (lane == 0) ps.red[warp * kNPart] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kWarps; ++w) t += ps.red[w * kNPart];
    part_out[0] = t;
  }
}

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
  PhaseSmem<T> ps;
  double red[kNPart];
  int prefix[kMaxBatch + 1];
  int bail;
};

// Persistent cooperative kernel: every round, every CTA takes its share of
// the tiles of all active solves, runs for each solve the state transition
// and the decided phase, and then meets the others at one grid barrier.
template <typename T>
__global__ void __launch_bounds__(kThreads) k_ftgcr_persistent(BatchArgs<T> a) {
  extern __shared__ __align__(16) unsigned char dsm[];
  __shared__ KernelSmem<T> ks;
  T* sm = reinterpret_cast<T*>(dsm);
  double* smd = reinterpret_cast<double*>(dsm);
  const long long round0 = a.ctl->round0;
  const unsigned long long t_start = globaltimer();
  unsigned int nbar = 0;
  int it = 0;
  for (; it < a.max_rounds; ++it) {
    // watchdog: a kernel that runs far longer than any solve raises the error
    // flag; every CTA leaves at its next barrier
    if (threadIdx.x == 0 && globaltimer() - t_start > kKernelTimeoutNs) atomicExch(&a.ctl->err, 2);
    const long long round = round0 + it;
    const int par = (int)(round & 1);
    // tile prefix over active solves (identical in every CTA)
    if (threadIdx.x == 0) {
      int acc = 0;
      for (int s = 0; s < a.n; ++s) {
        const int act = __ldcg(a.active + par * a.n + s);
        ks.prefix[s] = acc;
        acc += act ? a.nt[s] : 0;
        if (!act && blockIdx.x == 0) a.active[(par ^ 1) * a.n + s] = 0;
      }
      ks.prefix[a.n] = acc;
    }
    __syncthreads();
    const int total = ks.prefix[a.n];
    if (total == 0) break;
    int cur = -1;
    for (int item = blockIdx.x; item < total; item += gridDim.x) {
      int lo = 0, hi = a.n - 1;  // last s with prefix[s] <= item and nt > 0
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (ks.prefix[mid] <= item) lo = mid; else hi = mid - 1;
      }
      const int s = lo;
      const int tau = item - ks.prefix[s];
      if (s != cur) {
        SolveDev<T>* sdp = a.solves[s];
        cta_load_cg(&ks.sd, sdp);
        __syncthreads();
        cta_load_cg(&ks.S, ks.sd.st + par);
        __syncthreads();
        reduce_partials(ks.sd.part + (long long)(par ^ 1) * ks.sd.nt * kNPart, ks.sd.nt,
                        part_count(ks.S.pending, ks.S.nu), ks.red);
        __syncthreads();
        if (threadIdx.x == 0) transition(ks.sd, ks.S, ks.red, ks.N, ks.c);
        __syncthreads();
        cur = s;
      }
      double* part_out = ks.sd.part + ((long long)par * ks.sd.nt + tau) * kNPart;
      switch (ks.c.kind) {
        case K_INIT: phase_init(ks.sd, ks.c, tau, sm, ks.ps, part_out); break;
        case K_PA: phase_pa(ks.sd, ks.c, tau, sm, ks.ps, part_out); break;
        case K_PB: phase_pb(ks.sd, ks.c, tau, ks.ps, part_out); break;
        case K_RESTORE: phase_restore(ks.sd, ks.c, tau, ks.ps, part_out); break;
        case K_OUT: phase_out(ks.sd, ks.c, tau, smd, ks.ps, part_out); break;
        case K_FIN: phase_fin(ks.sd, ks.c, tau, ks.ps, part_out); break;
        default: break;
      }
      __syncthreads();
      if (tau == 0) {
        cta_store(ks.sd.st + (par ^ 1), &ks.N);
        if (!ks.N.active) cta_store(ks.sd.result, &ks.N);
        if (threadIdx.x == 0) a.active[(par ^ 1) * a.n + s] = ks.N.active;
      }
      __syncthreads();
    }
    ++nbar;
    if (!grid_barrier(&a.ctl->counter, nbar * gridDim.x, &a.ctl->err, &ks.bail)) return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) a.ctl->round_end = round0 + it;
}

}  // namespace ftgcr
