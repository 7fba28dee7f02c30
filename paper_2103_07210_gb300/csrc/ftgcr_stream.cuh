// Streamed step rounds of the mixed path (FP32 inner vectors), for solves
// whose vectors live in HBM.
//
// A streamed solve gives each CTA one tall band of latitude rows (at most 64)
// and walks the band row by row.  For row j, the step's axpy (with the
// previous step's direction recurrences fused in, as in the PF round) reads
// its operand rows in chunks of 1024 columns through a ring of two or three
// shared-memory stage buffers: every thread copies its own four columns of
// each operand row with 16-byte cp.async, one or two stages ahead of the
// arithmetic, and later reads exactly those, so HBM traffic stays in flight
// without holding registers and a stage needs no barrier of its own.  r'
// lands in a row buffer; the row's zonal line solve (all eight warps on the
// one row, each lane on a contiguous piece; its constants arrive by bulk
// copies on an mbarrier while the axpy runs) turns it into e, which is
// written out and kept: three e rows stay in shared memory, so once e of row
// j exists the stencil L(e) of row j-1 and its dots stream their own operands
// (face coefficients, r', the L(p^l)) through the same ring.  Only the band's
// first and last rows need an e row of a neighbouring band; their stencils
// run in a second pass after a grid barrier.  No row is recomputed as halo
// and e is read back only at band edges, so a step moves about its
// algorithmic bytes (the line solve's constants, three rows per row, come on
// top).  Rows in shared memory are piece-major: lane l's C-element piece of
// the row is contiguous, padded to a pitch of C + 4 floats.
//
// Every wait on an mbarrier is bounded; a wait that runs out raises the
// launch's error flag, waits (bounded) for the copies still in flight, and the
// phase returns, so that the kernel leaves at its next grid barrier.
#pragma once

namespace ftgcr {

constexpr int kCW = 1024;                      // columns per chunk: one float4 per thread
constexpr int kMaxStreamRows = 64;             // rows of a streamed band
constexpr int kMaxRowList = 2 * kMaxStreamRows + 4;
constexpr unsigned long long kStreamWaitNs = 2000000000ull;  // 2 s per wait
constexpr unsigned long long kDrainNs = 500000000ull;        // 0.5 s for the copies left after a failure

// Per-CTA state of the streamed phases, in static shared memory of the
// streamed kernel instance only (no other instance refers to it).
struct StreamSmem {
  unsigned long long cfull;            // the line-solve constants of the next row
  unsigned int cph;                    // the parity cfull's next completion will show
  int bad;                             // a wait ran out
  int nrl;                             // entries of rl
  int rl[kMaxRowList];                 // the pass's row stages: (row << 1) | (0 axpy + line solve, 1 stencil)
  const float* tab_ax[4 + 2 * kMaxK];  // operand rows of an axpy stage
  const float* tab_st[4 + kMaxK];      // operand rows of a stencil stage (Ty - nlon: the south faces)
  float* out[5];                       // p', L(p'), r', phi', L(e) of this step
  float alpha[kMaxK];
  float beta;
  float muA[kMaxStreamRows];           // mu A_j of the band's rows
  float maps[kWarps * 64 + 2];         // line-solve piece maps, then y_0 and y_{m-1}
};
static __shared__ StreamSmem g_ss;

// ---- PTX: mbarriers, bulk copies, proxy fences
__device__ __forceinline__ void mbar_init(unsigned a, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(a), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned a, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(a), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned a, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(a), "r"(parity)
      : "memory");
  return ok != 0u;
}
// Wait for the phase of parity `parity` to complete, for at most `limit_ns`.
__device__ __forceinline__ bool mbar_wait(unsigned a, unsigned parity, unsigned long long limit_ns = kStreamWaitNs) {
  if (mbar_try(a, parity)) return true;
  const unsigned long long t0 = globaltimer();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(a, parity)) return true;
    if ((it & 31u) == 0u && globaltimer() - t0 > limit_ns) return false;
  }
}
// Global -> shared bulk copy completing on an mbarrier (16-byte aligned
// addresses, a multiple of 16 bytes).
__device__ __forceinline__ void bulk_load(unsigned dst, const void* src, unsigned bytes, unsigned mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}
// Orders this thread's generic-proxy view of global memory before its later
// bulk copies (which read through the async proxy).
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ V16<float> lds4(unsigned a) {
  V16<float> r;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(r.v[0]), "=f"(r.v[1]), "=f"(r.v[2]), "=f"(r.v[3])
               : "r"(a));
  return r;
}

// 16-byte global -> shared copy of this thread's columns.  No compiler memory
// clobber: the stage's data are read only after cp.async.wait_group, which
// carries one, and the rows copied are never written within the same stage.
__device__ __forceinline__ void cp_async16_nc(unsigned smem, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem), "l"(gmem));
}
__device__ __forceinline__ void sts_nc(unsigned a, float v) { asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v)); }

// Once per launch of the streamed instance, before any phase: the barriers.
__device__ __forceinline__ void stream_init() {
  if (threadIdx.x == 0) {
    mbar_init(smem_addr(&g_ss.cfull), 1);
    g_ss.cph = 0u;
    g_ss.bad = 0;
    fence_mbar_init();
  }
  __syncthreads();
}

// ---- piece-major rows
// The streamed rounds keep a row in shared memory piece-major: the row's 32
// per-lane chunks of C elements (C = sd.C, a power of two, lcb = log2 C) one
// after another with 4 floats of padding, element i at
// (i >> lcb) * (C + 4) + (i & (C - 1)).  Four consecutive columns starting at
// a multiple of 4 are then contiguous and 16-byte aligned, and the line
// solve's pieces (C / 8 consecutive elements of one lane chunk per thread)
// are read and written as float4 without bank conflicts (the chunk pitch
// C + 4 is an odd number of float4 words).  The line-solve constants of a
// streamed solve (c = -u, 1/w, z) come in the same layout (sd.lcp, lwp, lzp).
__device__ __forceinline__ int pk(int i, int lcb, int P) { return (i >> lcb) * P + (i & ((1 << lcb) - 1)); }
__device__ __forceinline__ void sts4(unsigned a, const V16<float>& v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.v[0]), "f"(v.v[1]), "f"(v.v[2]), "f"(v.v[3]));
}

// Periodic tridiagonal solve of row j (M e = -r, the zonal line
// preconditioner) in place in a piece-major row, by the whole block: thread
// (w, lane) takes elements lane * C + w * CP + kk, kk < CP = C / 8, held in
// registers.  Each recurrence of the leading block's factorisation (forward
// g_i = b_i + c_{i-1} g_{i-1}, b = -r; backward y_i = winv_i g_i + c_i y_{i+1})
// runs as: every piece's affine map, the maps of a lane's 8 pieces composed
// through shared memory, a warp scan over the lanes for each lane's carry-in,
// then each piece replayed from its exact carry-in.  The periodic coupling is
// eliminated by bordering with z: x_{n-1} = (b_{n-1} + Tx_{n-1} y_0 +
// Tx_{n-2} y_{m-1}) / delta, x_i = y_i - x_{n-1} z_i.  rb, cb, cw, cz: shared
// addresses of the row and of its constants; maps: 2 * 8 * 32 + 2 floats.
template <int CP>
__device__ __noinline__ void line_solve_piece(const SolveDev<float>& sd, int j, unsigned rb, unsigned cb, unsigned cw,
                                              unsigned cz, float* maps) {
  constexpr int G = kWarps;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int n = sd.nlon, m = n - 1, C = CP * G, P = C + 4, lcb = __ffs(C) - 1;
  const unsigned base = 4u * (unsigned)(lane * P + w * CP);
  const int i0 = lane * C + w * CP;
  const float* lr = sd.lrow + (long long)j * 4;
  const float lr0 = __ldg(lr + 0), lr1 = __ldg(lr + 1), lr2 = __ldg(lr + 2);
  float* mF = maps;
  float* mG = maps + 32 * G;
  const float bl = -lds<float>(rb + 4u * (unsigned)pk(n - 1, lcb, P));
  // the forward multiplier of the piece's first element: c of the element before
  float a0 = 0.f;
  if (w > 0)
    a0 = lds<float>(cb + base - 4u);
  else if (lane > 0)
    a0 = lds<float>(cb + 4u * (unsigned)((lane - 1) * P + C - 1));
  float r[CP], cv[CP];
#pragma unroll
  for (int q = 0; q < CP; q += 4) {
    const V16<float> x = lds4(rb + base + 4u * q), y = lds4(cb + base + 4u * q);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      // positions past the row hold no data (their factors are zero)
      r[q + u] = i0 + q + u < n ? x.v[u] : 0.f;
      cv[q + u] = y.v[u];
    }
  }
  // forward: the piece's map g_out = F g_in + Gm
  float F = 1.f, Gm = 0.f;
  {
    float a = a0;
#pragma unroll
    for (int q = 0; q < CP; ++q) {
      Gm = fmaf(a, Gm, -r[q]);
      F = F * a;
      a = cv[q];
    }
  }
  mF[w * 32 + lane] = F;
  mG[w * 32 + lane] = Gm;
  __syncthreads();
  float FL = 1.f, GL = 0.f, Fw[G], Gw[G];
#pragma unroll
  for (int q = 0; q < G; ++q) {
    Fw[q] = mF[q * 32 + lane];
    Gw[q] = mG[q * 32 + lane];
    GL = fmaf(Fw[q], GL, Gw[q]);
    FL = FL * Fw[q];
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Fo = __shfl_up_sync(0xffffffffu, FL, d);
    const float Go = __shfl_up_sync(0xffffffffu, GL, d);
    if (lane >= d) {
      GL = fmaf(FL, Go, GL);
      FL = FL * Fo;
    }
  }
  float carry = __shfl_up_sync(0xffffffffu, GL, 1);
  if (lane == 0) carry = 0.f;
#pragma unroll
  for (int q = 0; q < G; ++q)
    if (q < w) carry = fmaf(Fw[q], carry, Gw[q]);
  {
    float a = a0, g = carry;
#pragma unroll
    for (int q = 0; q < CP; ++q) {
      g = fmaf(a, g, -r[q]);
      r[q] = g;
      a = cv[q];
    }
  }
  __syncthreads();  // every carry read before the maps are reused
  // backward: the piece's map y_in = Fb y_out + Y
  float wv[CP];
#pragma unroll
  for (int q = 0; q < CP; q += 4) {
    const V16<float> y = lds4(cw + base + 4u * q);
#pragma unroll
    for (int u = 0; u < 4; ++u) wv[q + u] = y.v[u];
  }
  float Fb = 1.f, Y = 0.f;
#pragma unroll
  for (int q = CP - 1; q >= 0; --q) {
    Y = fmaf(cv[q], Y, r[q] * wv[q]);
    Fb = Fb * cv[q];
  }
  mF[w * 32 + lane] = Fb;
  mG[w * 32 + lane] = Y;
  __syncthreads();
  float FbL = 1.f, YL = 0.f;
#pragma unroll
  for (int q = G - 1; q >= 0; --q) {
    Fw[q] = mF[q * 32 + lane];
    Gw[q] = mG[q * 32 + lane];
    YL = fmaf(Fw[q], YL, Gw[q]);
    FbL = FbL * Fw[q];
  }
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const float Fo = __shfl_down_sync(0xffffffffu, FbL, d);
    const float Yo = __shfl_down_sync(0xffffffffu, YL, d);
    if (lane + d < 32) {
      YL = fmaf(FbL, Yo, YL);
      FbL = FbL * Fo;
    }
  }
  float carryb = __shfl_down_sync(0xffffffffu, YL, 1);
  if (lane == 31) carryb = 0.f;
#pragma unroll
  for (int q = G - 1; q >= 0; --q)
    if (q > w) carryb = fmaf(Fw[q], carryb, Gw[q]);
  {
    float y = carryb;
#pragma unroll
    for (int q = CP - 1; q >= 0; --q) {
      y = fmaf(cv[q], y, r[q] * wv[q]);
      r[q] = y;
    }
  }
  // bordering: y_0 and y_{m-1} from the threads that hold them
  if (i0 == 0) maps[64 * G] = r[0];
#pragma unroll
  for (int q = 0; q < CP; ++q)
    if (i0 + q == m - 1) maps[64 * G + 1] = r[q];
  __syncthreads();
  const float y0 = maps[64 * G], ym = maps[64 * G + 1];
  const float xl = fmaf(lr2, ym, fmaf(lr1, y0, bl * lr0));
#pragma unroll
  for (int q = 0; q < CP; q += 4) {
    const V16<float> z = lds4(cz + base + 4u * q);
    V16<float> o;
#pragma unroll
    for (int u = 0; u < 4; ++u) o.v[u] = fmaf(-xl, z.v[u], r[q + u]);
    sts4(rb + base + 4u * q, o);
  }
  __syncthreads();
  if (threadIdx.x == 0) sts(rb + 4u * (unsigned)pk(n - 1, lcb, P), xl);
  __syncthreads();
}

// ---- the ring of stage buffers
// A stage is one chunk of kCW columns of one row stage: an axpy stage reads
// L(e), r, e, phi, then L(p^l), p^l for l = 0..nu_o (fused, PF) or L(p^nu),
// r, p^nu, phi (PA); a stencil stage reads Tx, Ty (north face), Ty of the row
// below (south face), r', then L(p^l) for l = 0..nu.  A stage with more than
// kNVS operand rows is taken in sub-stages of kNVS.  Thread t copies, with
// 16-byte cp.async, columns 4t .. 4t+3 of each operand row of the chunk into
// the stage buffer and later reads exactly those, so a stage needs no
// cross-thread synchronisation; lane 0 of each warp also copies the Tx
// element west of its warp's columns.  sd.nslot stage buffers are used in
// turn, sd.nslot - 1 stages ahead of the arithmetic.
constexpr int kNVS = 12;  // operand rows per (sub-)stage

__device__ __forceinline__ void cp_async_wait_n(int n) {
  if (n <= 0)
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  else if (n == 1)
    asm volatile("cp.async.wait_group 1;" ::: "memory");
  else
    asm volatile("cp.async.wait_group 2;" ::: "memory");
}

// Operand row v of an axpy stage.
template <bool FUSED>
__device__ __forceinline__ const float* ax_src(const Ctx<float>& c, int v) {
  if constexpr (FUSED) {
    if (v == 0) return c.LeR;
    if (v == 1) return c.rC;
    if (v == 2) return c.eR;
    if (v == 3) return c.phiC;
    const int l = (v - 4) >> 1;
    return ((v - 4) & 1) ? c.pp[l] : c.lo[l];
  } else {
    if (v == 0) return c.lpnu;
    if (v == 1) return c.rC;
    if (v == 2) return c.pnu;
    return c.phiC;
  }
}
// This thread's copies of (sub-)stage `sub` of chunk ch of a row stage into
// stage buffer `buf` (shared address), and, for a stencil stage, lane 0's
// copy of the Tx element west of its warp's columns into `lead`.  The
// operand rows come from the pass's tables (tab: axpy or stencil).
__device__ __forceinline__ void stream_copy(const float* const* tab, const float* Tx, int n, int nlat, int type,
                                            int row, int ch, int sub, int nv, unsigned buf, unsigned lead) {
  const int c0 = ch * kCW, i4 = 4 * (int)threadIdx.x;
  const long long ro = (long long)row * n;
  const int v0 = sub * kNVS;
  if (type == 1 && sub == 0 && (threadIdx.x & 31) == 0) {
    const int w0 = c0 + 128 * (int)(threadIdx.x >> 5);
    if (w0 < n) cp_async16_nc(lead + 16u * (threadIdx.x >> 5), Tx + ro + (w0 >= 4 ? w0 - 4 : n - 4));
  }
  if (c0 + i4 >= n) return;
  const long long off = ro + c0 + i4;
#pragma unroll
  for (int q = 0; q < kNVS; ++q) {
    const int v = v0 + q;
    // pole rows have no north (last row) or south (first row) face
    const bool face = type == 0 || !((v == 1 && row == nlat - 1) || (v == 2 && row == 0));
    if (v < nv && face) cp_async16_nc(buf + 4u * (unsigned)(q * kCW + i4), tab[v] + off);
  }
}

// Registers an axpy stage carries across its sub-stages.
struct AxRegs {
  V16<float> ln, rr, pn, ph;
};

// Sub-stage `sub` of an axpy chunk (the same operations, in the same order, as
// the PA / PF axpy of the other round layouts).  After the last sub-stage:
// the flips of the step, r'' and phi'', the norm, the state vectors of the
// row written, r'' into the row buffer.
template <bool FUSED>
__device__ __forceinline__ void stream_ax(int n, int lcb, int P, const PhaseSmem& ps, unsigned buf, int row, int ch,
                                          int sub, int nv, unsigned rb, AxRegs& x, Acc<float>& an) {
  const int c0 = ch * kCW, i4 = 4 * (int)threadIdx.x;
  if (c0 + i4 >= n) return;
  const int v0 = sub * kNVS;
  auto S = [&](int q) { return lds4(buf + 4u * (unsigned)(q * kCW + i4)); };
  if (sub == 0) {
    x.ln = S(0);
    x.rr = S(1);
    x.pn = S(2);
    x.ph = S(3);
  }
  if constexpr (FUSED) {
#pragma unroll
    for (int q = 0; q < kNVS; q += 2) {
      const int v = v0 + q;
      if (v >= 4 && v < nv) {
        const float al = g_ss.alpha[(v - 4) >> 1];
        const V16<float> ll = S(q), pl = S(q + 1);
#pragma unroll
        for (int w = 0; w < 4; ++w) {
          x.ln.v[w] = fmaf(al, ll.v[w], x.ln.v[w]);
          x.pn.v[w] = fmaf(al, pl.v[w], x.pn.v[w]);
        }
      }
    }
  }
  if (v0 + kNVS < nv) return;  // more sub-stages to come
  const long long g = (long long)row * n + c0 + i4;
  const float beta = g_ss.beta;
  const int nfl = ps.nfl;
  V16<float> rn, fn;
  if constexpr (FUSED) {
    if (nfl) {
#pragma unroll
      for (int w = 0; w < 4; ++w) {
        x.rr.v[w] = apply_flips(x.rr.v[w], g + w, V_R, nfl, ps.fl);
        x.ln.v[w] = apply_flips(x.ln.v[w], g + w, V_AP, nfl, ps.fl);
        x.ph.v[w] = apply_flips(x.ph.v[w], g + w, V_X, nfl, ps.fl);
        x.pn.v[w] = apply_flips(x.pn.v[w], g + w, V_P, nfl, ps.fl);
      }
    }
  }
  // plain (PA): ln holds L(p^nu), pn holds p^nu
#pragma unroll
  for (int w = 0; w < 4; ++w) {
    rn.v[w] = fmaf(beta, x.ln.v[w], x.rr.v[w]);
    fn.v[w] = fmaf(beta, x.pn.v[w], x.ph.v[w]);
    an.add(rn.v[w], rn.v[w]);
  }
  if constexpr (FUSED) {
    stv(g_ss.out[0] + g, x.pn);
    stv(g_ss.out[1] + g, x.ln);
  }
  stv(g_ss.out[2] + g, rn);
  stv(g_ss.out[3] + g, fn);
  sts4(rb + 4u * (unsigned)pk(c0 + i4, lcb, P), rn);
}

// Registers a stencil stage carries across its sub-stages.
struct StRegs {
  V16<float> le;
};

// Sub-stage `sub` of a stencil chunk of row `row`: (sub-stage 0) L(e) from the
// three e rows in shared memory (eC the row, eN north, eS south), written
// out, <r', L(e)> and <L(e), L(e)>, and e of the row written to eout unless
// it is null; (every sub-stage) the dots <L(e), L(p^l)> of its operand rows.  The operations of the stencil step of the other
// round layouts.
template <int KB>
__device__ __forceinline__ void stream_st(int n, int nlat, int lcb, int P, unsigned buf, unsigned lead, int row,
                                          int ch, int sub, int nv, unsigned eC, unsigned eN, unsigned eS, float muA,
                                          StRegs& x, Acc<float>* ad, Acc<float>& ah, Acc<float>& aq, float* eout) {
  const int c0 = ch * kCW, i4 = 4 * (int)threadIdx.x;
  const int v0 = sub * kNVS, v1 = min(nv, v0 + kNVS);
  const bool act = c0 + i4 < n;
  auto S = [&](int v) { return lds4(buf + 4u * (unsigned)((v - v0) * kCW + i4)); };
  if (sub == 0) {
    V16<float> tx;
    if (act) tx = S(0);
    // the element west of this thread's columns: the previous lane's last,
    // or for lane 0 the copy of its warp's lead
    float txw0 = __shfl_up_sync(0xffffffffu, act ? tx.v[3] : 0.f, 1);
    if ((threadIdx.x & 31) == 0 && act) txw0 = lds<float>(lead + 16u * (threadIdx.x >> 5) + 12u);
    if (!act) return;
    const bool hasN = row < nlat - 1, hasS = row > 0;
    V16<float> ty, tys;
    if (hasN) ty = S(1);
    if (hasS) tys = S(2);
    // e of the four columns, their north and south rows, and the columns
    // west of the first and east of the last (periodic)
    const int i = c0 + i4;
    const unsigned o = 4u * (unsigned)pk(i, lcb, P);
    const V16<float> ec = lds4(eC + o);
    if (eout) stv(eout + (long long)row * n + i, ec);
    V16<float> en, es;
    if (hasN) en = lds4(eN + o);
    if (hasS) es = lds4(eS + o);
    const float ew = lds<float>(eC + 4u * (unsigned)pk(i == 0 ? n - 1 : i - 1, lcb, P));
    const float ee = lds<float>(eC + 4u * (unsigned)pk(i + 4 == n ? 0 : i + 4, lcb, P));
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const float ve = w < 3 ? ec.v[w + 1] : ee;
      const float vw = w > 0 ? ec.v[w - 1] : ew;
      x.le.v[w] = stencil5<float>(ec.v[w], ve, vw, hasN ? en.v[w] : 0.f, hasS ? es.v[w] : 0.f, tx.v[w],
                                  w == 0 ? txw0 : tx.v[w - 1], hasN ? ty.v[w] : 0.f, hasS ? tys.v[w] : 0.f, muA, hasN,
                                  hasS);
    }
    stv(g_ss.out[4] + (long long)row * n + c0 + i4, x.le);
  }
  if (!act) return;
  // the dots with the L(p^l) of this sub-stage (static indices: the
  // accumulators stay in registers)
#pragma unroll
  for (int l = 0; l < KB; ++l) {
    const int v = 4 + l;
    if (v >= v0 && v < v1) {
      const V16<float> lp = S(v);
#pragma unroll
      for (int w = 0; w < 4; ++w) ad[l].add(x.le.v[w], lp.v[w]);
    }
  }
  if (sub == 0) {
    const V16<float> rn = S(3);
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      ah.add(rn.v[w], x.le.v[w]);
      aq.add(x.le.v[w], x.le.v[w]);
    }
  }
}

// Row j of a vector into a piece-major row (float4 accesses) and back.
__device__ __forceinline__ void stage_piece_row(const float* src, int j, int n, int lcb, int P, unsigned dst) {
  const float* s = src + (long long)j * n;
  for (int i = 4 * (int)threadIdx.x; i < n; i += 4 * kThreads) sts4(dst + 4u * (unsigned)pk(i, lcb, P), ldv(s + i));
}
__device__ __forceinline__ void store_piece_row(float* dst, int j, int n, int lcb, int P, unsigned src) {
  float* d = dst + (long long)j * n;
  for (int i = 4 * (int)threadIdx.x; i < n; i += 4 * kThreads) stv(d + i, lds4(src + 4u * (unsigned)pk(i, lcb, P)));
}
// The data-loss events of step t (Section 3) on e of row j in a piece-major
// row buffer (the flips of apply_losses that land in the row).
__device__ __forceinline__ void apply_losses_piece(const SolveDev<float>& sd, long long t, int j, float* row, int lcb,
                                                   int P) {
  const int nlon = sd.nlon;
  const long long g0 = (long long)j * nlon, g1 = g0 + nlon;
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
      unsigned int* w = reinterpret_cast<unsigned int*>(row + pk((int)(g - g0), lcb, P));
      atomicXor(w, 1u << (unsigned)((z >> 32) % 32u));
    }
  }
}

// Adds the CTA's sums of values [v0, nv) to the tile's partial sums already
// in `out` (FP32 path: one double per value).
__device__ __forceinline__ void cta_red_finish_add(CtaRed& cr, int nv, double* out, int v0) {
  __syncthreads();
  if (threadIdx.x >= v0 && threadIdx.x < nv) {
    const int v = threadIdx.x;
    double t[kWarps];
#pragma unroll
    for (int w = 0; w < kWarps; ++w) t[w] = cr.w[w][v].hi + cr.w[w][v].lo;
#pragma unroll
    for (int h = 1; h < kWarps; h <<= 1)
#pragma unroll
      for (int w = 0; w + h < kWarps; w += 2 * h) t[w] = t[w] + t[w + h];
    out[2 * v] = out[2 * v] + t[0];
  }
}

// The step round (PA, or PF with FUSED) of band tau of a streamed solve.
// pass 0: every row's axpy, line solve and e, and the stencils of the rows
// whose neighbours are all in the band; partial sums 0 (||r'||^2) and the
// dots of those rows.  pass 1 (after a grid barrier): the stencils of the
// band's edge rows, with the neighbouring band's e row read back; their dots
// added to the partial sums.  Shared memory: three piece-major e rows
// (32 (C + 4) floats each), the constants c, 1/w, z of one row (the same
// layout), sd.nslot stage buffers of
// kNVS * kCW floats, then the Tx leads (sd.nslot x 8 x 16 bytes).
template <int KB, bool FUSED>
__device__ __noinline__ void phase_stream(const SolveDev<float>& sd, const Ctx<float>& c, int tau, float* sm,
                                          PhaseSmem& ps, double* part_out, int pass, int* err) {
  const int n = sd.nlon, nlat = sd.nlat, C = sd.C, P = C + 4, lcb = __ffs(C) - 1;
  const int stride = 32 * P;  // a piece-major row
  const int j0 = row_start(nlat, sd.nt, tau), j1 = row_start(nlat, sd.nt, tau + 1);
  const int nch = (n + kCW - 1) / kCW, nbuf = sd.nslot, D = nbuf - 1;
  const int nv_ax = FUSED ? 4 + 2 * (c.nuo + 1) : 4;
  const int nv_st = 5 + c.nu;
  const int ns_ax = (nv_ax + kNVS - 1) / kNVS, ns_st = (nv_st + kNVS - 1) / kNVS;
  float* ebuf = sm;
  float* cst = sm + 3 * stride;
  const unsigned cst_s = smem_addr(cst);
  float* ring = cst + 3 * stride;
  const unsigned ring_s = smem_addr(ring);
  const unsigned lead_s = smem_addr(ring + (size_t)nbuf * kNVS * kCW);
  const unsigned per = 4u * (unsigned)stride;  // bytes of one constants row
  auto interior = [&](int i) { return (i == 0 || i - 1 >= j0) && (i == nlat - 1 || i + 1 < j1); };
  if (threadIdx.x == 0) {
    ps.cs_solve = -1;  // the dynamic shared memory is laid out for this phase
    int m = 0;
    if (pass == 0) {
      for (int j = j0; j < j1; ++j) {
        g_ss.rl[m++] = j << 1;
        if (j - 1 >= j0 && interior(j - 1)) g_ss.rl[m++] = ((j - 1) << 1) | 1;
      }
      if (j1 == nlat && j1 - 1 >= j0 && interior(j1 - 1)) g_ss.rl[m++] = ((j1 - 1) << 1) | 1;
      ps.nfl = collect_flips(sd, c.t, FUSED ? (kStateVecs | (1u << V_E)) : (1u << V_E), (long long)j0 * n,
                             (long long)j1 * n, ps.fl);
    } else {
      if (!interior(j0)) g_ss.rl[m++] = (j0 << 1) | 1;
      if (j1 - 1 != j0 && !interior(j1 - 1)) g_ss.rl[m++] = ((j1 - 1) << 1) | 1;
    }
    g_ss.nrl = m;
  }
  if ((int)threadIdx.x < j1 - j0) g_ss.muA[threadIdx.x] = __ldg(sd.muA + j0 + threadIdx.x);
  // the pass's operand tables, outputs and coefficients
  if ((int)threadIdx.x < nv_ax) g_ss.tab_ax[threadIdx.x] = ax_src<FUSED>(c, threadIdx.x);
  if ((int)threadIdx.x >= 64 && (int)threadIdx.x < 64 + nv_st) {
    const int v = threadIdx.x - 64;
    g_ss.tab_st[v] = v == 0 ? sd.Tx : v == 1 ? sd.Ty : v == 2 ? sd.Ty - n : v == 3 ? c.rW : c.lp[v - 4];
  }
  if ((int)threadIdx.x >= 128 && (int)threadIdx.x < 128 + kMaxK) g_ss.alpha[threadIdx.x - 128] = c.alpha[threadIdx.x - 128];
  if (threadIdx.x == 160) {
    g_ss.out[0] = c.pnew;
    g_ss.out[1] = c.lpnew;
    g_ss.out[2] = c.rW;
    g_ss.out[3] = c.phiW;
    g_ss.out[4] = c.LeW;
    g_ss.beta = c.beta;
  }
  __syncthreads();
  const int nrl = g_ss.nrl;
  unsigned cph = g_ss.cph;
  auto issue_consts = [&](int row) {  // thread 0: one row of c, 1/w, z by bulk copies
    const unsigned mb = smem_addr(&g_ss.cfull);
    const long long o = (long long)row * stride;
    mbar_expect(mb, 3u * per);
    bulk_load(cst_s, sd.lcp + o, per, mb);
    bulk_load(cst_s + per, sd.lwp + o, per, mb);
    bulk_load(cst_s + 2u * per, sd.lzp + o, per, mb);
  };
  if (threadIdx.x == 0 && pass == 0 && j0 < j1) {
    fence_proxy_async_global();
    issue_consts(j0);
  }
  // stage issue cursor (every thread the same): row stage, chunk, sub-stage
  int pi = 0, pc = 0, psb = 0, pidx = 0;
  auto issue_next = [&]() {
    if (pi < nrl) {
      const int e = g_ss.rl[pi], type = e & 1, row = e >> 1;
      const int b = pidx % nbuf;
      stream_copy(type ? g_ss.tab_st : g_ss.tab_ax, sd.Tx, n, nlat, type, row, pc, psb, type ? nv_st : nv_ax,
                  ring_s + 4u * (unsigned)(b * kNVS * kCW), lead_s + 128u * (unsigned)b);
      if (++psb == (type ? ns_st : ns_ax)) {
        psb = 0;
        if (++pc == nch) {
          pc = 0;
          ++pi;
        }
      }
    }
    cp_async_commit();  // an empty group once the pass is issued: the counts stay aligned
    ++pidx;
  };
  for (int d = 0; d < D; ++d) issue_next();
  Acc<float> an, ah, aq;
  Acc<float> ad[KB];
  int cidx = 0;
  bool fail = false;
  for (int ci = 0; ci < nrl; ++ci) {
    const int e = g_ss.rl[ci], type = e & 1, row = e >> 1;
    const int nv = type ? nv_st : nv_ax, ns = type ? ns_st : ns_ax;
    unsigned eC = 0, eN = 0, eS = 0;
    if (type == 1) {
      if (pass == 0) {
        eC = smem_addr(ebuf + (row % 3) * stride);
        eN = smem_addr(ebuf + ((row + 1) % 3) * stride);
        eS = smem_addr(ebuf + ((row + 2) % 3) * stride);
      } else {
        // the three e rows, the neighbour's included (plain loads; this row's
        // stage copies are in flight meanwhile)
        __syncthreads();  // the previous row's stencil has read them
        if (row > 0) stage_piece_row(c.eW, row - 1, n, lcb, P, smem_addr(ebuf));
        stage_piece_row(c.eW, row, n, lcb, P, smem_addr(ebuf + stride));
        if (row < nlat - 1) stage_piece_row(c.eW, row + 1, n, lcb, P, smem_addr(ebuf + 2 * stride));
        __syncthreads();
        eS = smem_addr(ebuf);
        eC = smem_addr(ebuf + stride);
        eN = smem_addr(ebuf + 2 * stride);
      }
    }
    // An axpy row needs no barrier here: it writes r' only at this thread's
    // columns of the buffer, whose last reader (the stencil two rows back, its
    // south row) read only this thread's columns.
    float* rowbuf = ebuf + (row % 3) * stride;
    const unsigned rb = smem_addr(rowbuf);
    const float muA = g_ss.muA[row - j0];
    for (int ch = 0; ch < nch; ++ch) {
      AxRegs xa;
      StRegs xs;
      for (int sb = 0; sb < ns; ++sb) {
        // the next stage's copies go out before this one is waited for; a
        // stage never reads a row this thread writes within the last D stages
        issue_next();
        cp_async_wait_n(D);
        const int b = cidx % nbuf;
        const unsigned buf = ring_s + 4u * (unsigned)(b * kNVS * kCW);
        if (type == 0)
          stream_ax<FUSED>(n, lcb, P, ps, buf, row, ch, sb, nv, rb, xa, an);
        else
          stream_st<KB>(n, nlat, lcb, P, buf, lead_s + 128u * (unsigned)b, row, ch, sb, nv, eC, eN, eS, muA, xs, ad,
                        ah, aq, pass == 0 ? c.eW : nullptr);
        ++cidx;
      }
    }
    if (type == 1) continue;
    // the row's line solve: e = P^-1 r' in place
    __syncthreads();  // r' of every column in the row buffer
    {
      bool ok = true;
      if ((threadIdx.x & 31) == 0) ok = mbar_wait(smem_addr(&g_ss.cfull), cph & 1u);
      if (!__shfl_sync(0xffffffffu, ok ? 1 : 0, 0)) g_ss.bad = 1;
      __syncwarp();
    }
    __syncthreads();
    if (g_ss.bad) {
      fail = true;
      break;
    }
    cph ^= 1u;
    {
      const unsigned cb = cst_s, cwb = cst_s + per, czb = cst_s + 2u * per;
      if (C == 32)
        line_solve_piece<4>(sd, row, rb, cb, cwb, czb, g_ss.maps);
      else if (C == 64)
        line_solve_piece<8>(sd, row, rb, cb, cwb, czb, g_ss.maps);
      else if (C == 128)
        line_solve_piece<16>(sd, row, rb, cb, cwb, czb, g_ss.maps);
      else
        line_solve_piece<32>(sd, row, rb, cb, cwb, czb, g_ss.maps);
    }
    if (threadIdx.x == 0) {
      // the constants are consumed: the next row's may come in
      if (row + 1 < j1) issue_consts(row + 1);
      for (int q = 0; q < ps.nfl; ++q) {  // e-site flips (the paper's injection site)
        if (ps.fl[q].vec != V_E) continue;
        const long long g = ps.fl[q].g;
        const int jj = (int)(g / n), i = (int)(g - (long long)jj * n);
        if (jj != row) continue;
        rowbuf[pk(i, lcb, P)] = flip_bits(rowbuf[pk(i, lcb, P)], ps.fl[q].bit);
      }
    }
    if (sd.nlosses) {
      __syncthreads();
      apply_losses_piece(sd, c.t, row, rowbuf, lcb, P);
    }
    if (ps.nfl || sd.nlosses) __syncthreads();  // thread 0's flips before any reader
    if (!interior(row)) store_piece_row(c.eW, row, n, lcb, P, rb);  // else stored by its stencil
  }
  cp_async_wait_all();  // the groups still open are empty unless the pass failed
  if (fail) {
    if (threadIdx.x == 0) {
      atomicExch(err, 3);
      // a constants copy may still be in flight: let it land (bounded)
      mbar_wait(smem_addr(&g_ss.cfull), cph & 1u, kDrainNs);
    }
    return;
  }
  if (pass == 0) {
    cta_red_put(ps.cr, 0, an.warp_sum());
#pragma unroll
    for (int l = 0; l < KB; ++l)
      if (l <= c.nu) cta_red_put(ps.cr, 1 + l, ad[l].warp_sum());
    cta_red_put(ps.cr, 2 + c.nu, ah.warp_sum());
    cta_red_put(ps.cr, 3 + c.nu, aq.warp_sum());
    cta_red_finish<float>(ps.cr, 4 + c.nu, part_out);
  } else {
#pragma unroll
    for (int l = 0; l < KB; ++l)
      if (l <= c.nu) cta_red_put(ps.cr, 1 + l, ad[l].warp_sum());
    cta_red_put(ps.cr, 2 + c.nu, ah.warp_sum());
    cta_red_put(ps.cr, 3 + c.nu, aq.warp_sum());
    cta_red_finish_add(ps.cr, 4 + c.nu, part_out, 1);
  }
  if (threadIdx.x == 0) g_ss.cph = cph;
}

}  // namespace ftgcr
