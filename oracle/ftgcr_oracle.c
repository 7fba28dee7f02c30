/*
 * FT-GCR(k) oracle: a plain, slow, sequential FP64 CPU implementation of what
 * the GPU library computes.  TEST INFRASTRUCTURE ONLY: it may be used by the
 * tests, by the package's smoke check and by the CPU-baseline leg of the
 * benchmark, never by the product path.  It shares no code, header, table or
 * constant with the CUDA library.
 *
 * Paper: M. Gillard, T. Benacchio, "FT-GCR: a fault-tolerant generalized
 * conjugate residual elliptic solver" (arXiv 2103.07210).
 *
 *  - Problem:   L(phi) = R, Eq. (1), Section 2.  The paper's operator is a 3-D
 *               terrain-following Poisson operator on octahedral grids
 *               (Section 3, Eq. (3)); it gives no discrete formula.  This
 *               oracle uses the 2-D latitude-longitude finite-volume analogue
 *               (column depth D = 1 - h over a Gaussian hill, Section 3)
 *               with a Helmholtz term -mu*A*phi that makes -L definite.
 *  - Preconditioner: Section 2 only says "bespoke left-preconditioning" aimed
 *               at the anisotropy of global grids.  Reading used here: the
 *               zonal (longitude-line) part of L plus the diagonal of the
 *               rest, one periodic tridiagonal system per latitude row.
 *  - Iteration: Algorithm 1 (FT-GCR(k)), with these readings of the printed
 *               algorithm: beta and alpha_l carry a minus sign (with
 *               r = L(phi) - R the printed signs make ||r|| grow); the
 *               p/L(p) recurrences run after the l loop; the cycle end copies
 *               ^k into ^0; a detected fault aborts the cycle and restarts it
 *               from the backup; the backup also starts as ^0 after the
 *               initialisation; the fault test is !(new < old), i.e. ">=" for
 *               finite values, also true for NaN; norms are compared squared;
 *               the exit tolerance is relative to ||R||.
 *  - Faults:    Section 3 injects bit flips into e = P^-1(r).  Here a plan of
 *               single-bit flips {step, vector, index, bit} fires at the start
 *               of executed step `step` (x, r, p, Ap: before beta is formed)
 *               or right after the preconditioner of that step (e).
 *               Section 3's data-loss events are also modelled: at a given
 *               step, `count` entries of e inside one "process" block (the
 *               block `rank` of `nranks` equal contiguous blocks of the
 *               row-major array) each suffer one bit flip; entry and bit of
 *               flip i come from output i of SplitMix64 (Steele, Lea and
 *               Flood, 2014) started at the event's seed.
 *  - Protection: `protect` = 0 runs plain GCR(k) (the paper's unprotected
 *               runs): no fault test, no backup, no restore.
 *
 * Every reduction is a sequential sum in index order accumulated in twice the
 * working precision and rounded once (Dot2).  Every pointwise update is
 * written as an explicit fma where the method multiplies and adds (axpy,
 * recurrences, line-solve substitution); everything else uses separately
 * rounded operations (compile with -ffp-contract=off).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

enum { ORC_VEC_X = 0, ORC_VEC_R = 1, ORC_VEC_P = 2, ORC_VEC_AP = 3, ORC_VEC_E = 4 };
enum { ORC_PRECOND_LINE = 0, ORC_PRECOND_JACOBI = 1, ORC_PRECOND_IDENTITY = 2, ORC_PRECOND_DENSE = 3 };
enum { ORC_EVENT_ACCEPT = 0, ORC_EVENT_FAULT = 1, ORC_EVENT_EXIT = 2 };

typedef struct {
  int64_t step;  /* executed-step number (1-based, re-executed steps count) */
  int32_t vec;   /* ORC_VEC_* */
  int64_t index; /* element, row-major [nlat][nlon] */
  int32_t bit;   /* 0..63 of the IEEE-754 binary64 pattern */
} orc_fault;

typedef struct {
  int32_t nlon, nlat;
  double mu;             /* Helmholtz coefficient (per unit area) */
  int32_t k;             /* Krylov cycle length */
  double tol;            /* exit when ||r|| <= tol * ||R|| */
  int64_t max_steps;     /* executed-step limit */
  int32_t precond;       /* ORC_PRECOND_* */
  const double* D;       /* [nlat][nlon] cell-centred coefficient */
  const double* dense_pinv; /* [N][N] row-major, only for ORC_PRECOND_DENSE */
  int32_t protect;       /* 1: FT-GCR(k) (Algorithm 1); 0: plain GCR(k), no fault test */
} orc_problem;

/* One data-loss event (Section 3): at executed step `step`, right after the
 * preconditioner, `count` single-bit flips hit e inside block `rank` of
 * `nranks`: elements [floor(rank N / nranks), floor((rank + 1) N / nranks)).
 * Flip i (i = 1..count) takes z = output i of SplitMix64 started at `seed`,
 * element block_start + z mod block_len and bit (z >> 32) mod nbits. */
typedef struct {
  int64_t step;
  int32_t rank, nranks;
  int64_t count;
  uint64_t seed;
  int32_t nbits;
} orc_loss;

#define ORC_MAX_DETECT 64
typedef struct {
  int64_t steps, cycles, restarts, faults_injected, faults_detected;
  int64_t loss_events;     /* data-loss events that fired */
  int32_t converged, ndetect;
  int64_t detect_step[ORC_MAX_DETECT];
  double nrm2_R, nrm2_0, nrm2_final, res_true;
} orc_result;

/* ---------------------------------------------------------------- geometry */
/* Regular latitude-longitude grid on the unit sphere: cell (i, j) has centre
 * lambda_i = (i + 1/2) dlam, theta_j = -pi/2 + (j + 1/2) dth; the faces of row j
 * sit at theta_{j -+ 1/2}.  Per row: the east-west face factor
 * cx_j = dth / (cos(theta_j) dlam), the north face factor
 * cy_j = cos(theta_{j+1/2}) dlam / dth (zero at the north pole face) and the
 * exact cell area A_j = dlam (sin theta_{j+1/2} - sin theta_{j-1/2}). */
void orc_geometry(int nlon, int nlat, double* cx, double* cy, double* area) {
  double dlam = 2.0 * ORC_PI / nlon;
  double dth = ORC_PI / nlat;
  for (int j = 0; j < nlat; ++j) {
    double th = -0.5 * ORC_PI + (j + 0.5) * dth;
    double s_south = (j == 0) ? -1.0 : sin(-0.5 * ORC_PI + j * dth);
    double s_north = (j == nlat - 1) ? 1.0 : sin(-0.5 * ORC_PI + (j + 1) * dth);
    cx[j] = dth / (cos(th) * dlam);
    cy[j] = (j == nlat - 1) ? 0.0 : cos(-0.5 * ORC_PI + (j + 1) * dth) * dlam / dth;
    area[j] = dlam * (s_north - s_south);
  }
}

/* Face coefficients of the finite-volume operator: arithmetic mean of D on
 * each face times the face geometry.  Tx[j][i] is the face between (i, j) and
 * (i+1 mod nlon, j); Ty[j][i] the face between (i, j) and (i, j+1); the pole
 * faces carry no flux (Ty of the last row is zero, the south face of row 0 is
 * never used). */
void orc_face_coeffs(int nlon, int nlat, const double* D, double* Tx, double* Ty, double* area) {
  double* cx = (double*)malloc(sizeof(double) * nlat);
  double* cy = (double*)malloc(sizeof(double) * nlat);
  orc_geometry(nlon, nlat, cx, cy, area);
  for (int j = 0; j < nlat; ++j)
    for (int i = 0; i < nlon; ++i) {
      int ie = (i + 1) % nlon;
      Tx[(long)j * nlon + i] = 0.5 * (D[(long)j * nlon + i] + D[(long)j * nlon + ie]) * cx[j];
      Ty[(long)j * nlon + i] = (j == nlat - 1) ? 0.0 : 0.5 * (D[(long)j * nlon + i] + D[(long)(j + 1) * nlon + i]) * cy[j];
    }
  free(cx);
  free(cy);
}

/* ---------------------------------------------------------------- operator */
/* (L phi)_{j,i} = Tx_{j,i} (phi_{j,i+1} - phi_{j,i}) + Tx_{j,i-1} (phi_{j,i-1} - phi_{j,i})
 *              + Ty_{j,i} (phi_{j+1,i} - phi_{j,i}) + Ty_{j-1,i} (phi_{j-1,i} - phi_{j,i})
 *              - (mu A_j) phi_{j,i}
 * periodic in i; the north term is absent on the last row, the south term on
 * row 0.  Summed left to right in exactly this order. */
void orc_apply_L(int nlon, int nlat, double mu, const double* Tx, const double* Ty, const double* area,
                 const double* phi, double* out) {
  for (int j = 0; j < nlat; ++j) {
    double muA = mu * area[j];
    for (int i = 0; i < nlon; ++i) {
      long c = (long)j * nlon + i;
      long e = (long)j * nlon + (i + 1) % nlon;
      long w = (long)j * nlon + (i + nlon - 1) % nlon;
      double v = phi[c];
      double s = Tx[c] * (phi[e] - v) + Tx[w] * (phi[w] - v);
      if (j < nlat - 1) s = s + Ty[c] * (phi[c + nlon] - v);
      if (j > 0) s = s + Ty[c - nlon] * (phi[c - nlon] - v);
      out[c] = s - muA * v;
    }
  }
}

/* Preconditioner operator P: the zonal part of L plus the diagonal of the
 * meridional and Helmholtz parts,
 * (P phi)_{j,i} = Tx_{j,i} (phi_{j,i+1} - phi_{j,i}) + Tx_{j,i-1} (phi_{j,i-1} - phi_{j,i})
 *              - (Ty_{j,i} + Ty_{j-1,i} + mu A_j) phi_{j,i}. */
static double orc_sigma(int nlon, int nlat, const double* Ty, double muA, int j, int i) {
  double s = 0.0;
  if (j < nlat - 1) s = s + Ty[(long)j * nlon + i];
  if (j > 0) s = s + Ty[(long)(j - 1) * nlon + i];
  return s + muA;
}

void orc_apply_P(int nlon, int nlat, double mu, const double* Tx, const double* Ty, const double* area,
                 const double* phi, double* out) {
  for (int j = 0; j < nlat; ++j) {
    double muA = mu * area[j];
    for (int i = 0; i < nlon; ++i) {
      long c = (long)j * nlon + i;
      long e = (long)j * nlon + (i + 1) % nlon;
      long w = (long)j * nlon + (i + nlon - 1) % nlon;
      double v = phi[c];
      double s = Tx[c] * (phi[e] - v) + Tx[w] * (phi[w] - v);
      out[c] = s - orc_sigma(nlon, nlat, Ty, muA, j, i) * v;
    }
  }
}

/* Solve one periodic symmetric tridiagonal system M x = b of order n >= 3,
 * M_ii = d_i, M_{i,i+1} = M_{i+1,i} = -o_i (o_{n-1} couples x_{n-1} and x_0).
 * Textbook method: LU (Thomas) elimination of the leading (n-1) x (n-1) block
 * A0, with the periodic coupling of the last unknown eliminated by
 * bordering: x' = A0^-1 b' - x_{n-1} A0^-1 c, c = (-o_{n-1}, 0, ..., 0, -o_{n-2}),
 * and x_{n-1} from the last equation.
 *
 * Factorisation of A0 (sub_i = -o_{i-1}, sup_i = -o_i): w_0 = d_0,
 * l_i = sub_i / w_{i-1}, w_i = d_i - l_i sup_{i-1}; the pivots are kept as
 * reciprocals winv_i = 1 / w_i and u_i = sup_i winv_i.  Substitution:
 * forward y_i = b_i - l_i y_{i-1}, backward y_i = winv_i y_i - u_i y_{i+1},
 * each step one fused multiply-add. */
static void orc_thomas_factor(int m, const double* d, const double* o, double* l, double* winv, double* u) {
  double w = d[0];
  winv[0] = 1.0 / w;
  l[0] = 0.0;
  for (int i = 1; i < m; ++i) {
    l[i] = -o[i - 1] / w;
    w = d[i] - l[i] * -o[i - 1];
    winv[i] = 1.0 / w;
  }
  for (int i = 0; i < m; ++i) u[i] = (i < m - 1) ? -o[i] * winv[i] : 0.0;
}

static void orc_thomas_solve(int m, const double* l, const double* winv, const double* u, const double* rhs,
                             double* y) {
  y[0] = rhs[0];
  for (int i = 1; i < m; ++i) y[i] = fma(-l[i], y[i - 1], rhs[i]);
  y[m - 1] = y[m - 1] * winv[m - 1];
  for (int i = m - 2; i >= 0; --i) y[i] = fma(-u[i], y[i + 1], y[i] * winv[i]);
}

static void orc_periodic_tridiag(int n, const double* d, const double* o, const double* b, double* x,
                                 double* work) {
  int m = n - 1;
  double* l = work;
  double* winv = work + n;
  double* u = work + 2 * n;
  double* c = work + 3 * n;
  double* y = work + 4 * n;
  double* z = work + 5 * n;
  orc_thomas_factor(m, d, o, l, winv, u);
  for (int i = 0; i < m; ++i) c[i] = 0.0;
  c[0] = -o[n - 1];
  c[m - 1] = c[m - 1] + -o[n - 2];
  orc_thomas_solve(m, l, winv, u, b, y);
  orc_thomas_solve(m, l, winv, u, c, z);
  /* last row: -o_{n-1} x_0 - o_{n-2} x_{n-2} + d_{n-1} x_{n-1} = b_{n-1} */
  double num = b[n - 1] + o[n - 1] * y[0] + o[n - 2] * y[m - 1];
  double den = d[n - 1] + o[n - 1] * z[0] + o[n - 2] * z[m - 1];
  double xl = num / den;
  for (int i = 0; i < m; ++i) x[i] = y[i] - xl * z[i];
  x[n - 1] = xl;
}

/* e = P^-1 r for the preconditioner kinds of this oracle. */
void orc_solve_P(int nlon, int nlat, double mu, const double* Tx, const double* Ty, const double* area, int kind,
                 const double* dense_pinv, const double* r, double* e) {
  long N = (long)nlon * nlat;
  if (kind == ORC_PRECOND_IDENTITY) {
    for (long c = 0; c < N; ++c) e[c] = r[c];
    return;
  }
  if (kind == ORC_PRECOND_DENSE) {
    for (long a = 0; a < N; ++a) {
      double s = 0.0;
      for (long b = 0; b < N; ++b) s = s + dense_pinv[a * N + b] * r[b];
      e[a] = s;
    }
    return;
  }
  if (kind == ORC_PRECOND_JACOBI) {
    /* P = diag(L): L_cc = -(Tx_{j,i} + Tx_{j,i-1} + sigma_{j,i}) */
    for (int j = 0; j < nlat; ++j) {
      double muA = mu * area[j];
      for (int i = 0; i < nlon; ++i) {
        long c = (long)j * nlon + i;
        long w = (long)j * nlon + (i + nlon - 1) % nlon;
        double dg = Tx[c] + Tx[w] + orc_sigma(nlon, nlat, Ty, muA, j, i);
        e[c] = -r[c] / dg;
      }
    }
    return;
  }
  /* line preconditioner: P = -M row by row, so e = M^-1 (-r) */
  double* d = (double*)malloc(sizeof(double) * nlon);
  double* o = (double*)malloc(sizeof(double) * nlon);
  double* b = (double*)malloc(sizeof(double) * nlon);
  double* work = (double*)malloc(sizeof(double) * 6 * nlon);  /* l, winv, u, c, y, z */
  for (int j = 0; j < nlat; ++j) {
    double muA = mu * area[j];
    for (int i = 0; i < nlon; ++i) {
      long c = (long)j * nlon + i;
      long w = (long)j * nlon + (i + nlon - 1) % nlon;
      d[i] = Tx[c] + Tx[w] + orc_sigma(nlon, nlat, Ty, muA, j, i);
      o[i] = Tx[c];
      b[i] = -r[c];
    }
    orc_periodic_tridiag(nlon, d, o, b, e + (long)j * nlon, work);
  }
  free(d);
  free(o);
  free(b);
  free(work);
}

/* ------------------------------------------------------------ reductions */
/* Inner product accumulated in twice the working precision and rounded once
 * (Dot2 of Ogita, Rump and Oishi, 2005): each product split exactly into
 * h + r by one fma (TwoProduct), the running sum p advanced by Knuth's
 * TwoSum with its rounding error q, the low parts q + r collected in s,
 * result p + s. */
double orc_dot(long n, const double* a, const double* b) {
  double p = 0.0, s = 0.0;
  for (long i = 0; i < n; ++i) {
    double h = a[i] * b[i];
    double r = fma(a[i], b[i], -h);
    double t = p + h;
    double z = t - p;
    double q = (p - (t - z)) + (h - z);
    p = t;
    s = s + (q + r);
  }
  return p + s;
}

/* Flip one bit of the IEEE-754 binary64 pattern of v. */
double orc_flip_bit(double v, int bit) {
  uint64_t u;
  memcpy(&u, &v, sizeof u);
  u ^= (uint64_t)1 << bit;
  memcpy(&v, &u, sizeof v);
  return v;
}

static void orc_copy(long n, const double* a, double* b) { memcpy(b, a, sizeof(double) * n); }

/* Apply every fault of the plan that fires at executed step t on vector `vec`. */
static int orc_inject(const orc_fault* f, int nf, int64_t t, int vec, double* v, long N) {
  int fired = 0;
  for (int q = 0; q < nf; ++q)
    if (f[q].step == t && f[q].vec == vec && f[q].index >= 0 && f[q].index < N) {
      v[f[q].index] = orc_flip_bit(v[f[q].index], f[q].bit);
      ++fired;
    }
  return fired;
}

/* Output i (i >= 1) of SplitMix64 started at state `seed`: the state advances
 * by the golden-ratio increment 0x9E3779B97F4A7C15 per output and each output
 * is the state passed through the published finaliser (xor-shift 30, multiply
 * by 0xBF58476D1CE4E5B9, xor-shift 27, multiply by 0x94D049BB133111EB,
 * xor-shift 31). */
uint64_t orc_splitmix64(uint64_t seed, uint64_t i) {
  uint64_t z = seed + i * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

/* Apply every data-loss event of executed step t to e; returns how many fired. */
static int orc_data_loss(const orc_loss* ev, int nev, int64_t t, double* e, long N) {
  int fired = 0;
  for (int q = 0; q < nev; ++q) {
    if (ev[q].step != t || ev[q].nranks < 1 || ev[q].rank < 0 || ev[q].rank >= ev[q].nranks) continue;
    long b0 = (long)((int64_t)ev[q].rank * N / ev[q].nranks);
    long b1 = (long)((int64_t)(ev[q].rank + 1) * N / ev[q].nranks);
    long len = b1 - b0;
    if (len <= 0) continue;
    for (int64_t i = 1; i <= ev[q].count; ++i) {
      uint64_t z = orc_splitmix64(ev[q].seed, (uint64_t)i);
      long idx = b0 + (long)(z % (uint64_t)len);
      int bit = (int)((z >> 32) % (uint64_t)ev[q].nbits);
      e[idx] = orc_flip_bit(e[idx], bit);
    }
    ++fired;
  }
  return fired;
}

/* ------------------------------------------------------------- FT-GCR(k) */
/* Algorithm 1 of the paper with the readings listed at the top of this file.
 * x: in = initial guess phi^0, out = solution.  Optional per-step outputs
 * (length >= max_steps): nrm2_hist[t-1] = ||r^{nu+1}||^2 of step t,
 * event_hist[t-1] = ORC_EVENT_*, beta_hist[t-1] = beta.  lp_trace, if given,
 * receives L(p^nu) used by step t at lp_trace[(t-1)*N ...] (tiny grids only).
 * Returns 0 when converged, 1 when max_steps ran out, -1 on bad arguments. */
int orc_ftgcr(const orc_problem* pb, const double* R, double* x, const orc_fault* faults, int nfaults,
              const orc_loss* losses, int nlosses, orc_result* res, double* nrm2_hist, int32_t* event_hist,
              double* beta_hist, double* lp_trace) {
  int nlon = pb->nlon, nlat = pb->nlat, k = pb->k;
  if (nlon < 3 || nlat < 1 || k < 1 || !(pb->tol > 0.0)) return -1;
  long N = (long)nlon * nlat;
  memset(res, 0, sizeof *res);

  double* Tx = (double*)malloc(sizeof(double) * N);
  double* Ty = (double*)malloc(sizeof(double) * N);
  double* area = (double*)malloc(sizeof(double) * nlat);
  orc_face_coeffs(nlon, nlat, pb->D, Tx, Ty, area);

  /* state: phi, r (current), new phi, r, the cycle's directions p^0..p^k and
   * L(p^0)..L(p^k), e, L(e), and the backup [phi, r, p^0, L(p^0)]^* */
  double* phi = (double*)malloc(sizeof(double) * N);
  double* r = (double*)malloc(sizeof(double) * N);
  double* phin = (double*)malloc(sizeof(double) * N);
  double* rn = (double*)malloc(sizeof(double) * N);
  double* e = (double*)malloc(sizeof(double) * N);
  double* Le = (double*)malloc(sizeof(double) * N);
  double** p = (double**)malloc(sizeof(double*) * (k + 1));
  double** Lp = (double**)malloc(sizeof(double*) * (k + 1));
  for (int l = 0; l <= k; ++l) {
    p[l] = (double*)malloc(sizeof(double) * N);
    Lp[l] = (double*)malloc(sizeof(double) * N);
  }
  double* phi_s = (double*)malloc(sizeof(double) * N);
  double* r_s = (double*)malloc(sizeof(double) * N);
  double* p_s = (double*)malloc(sizeof(double) * N);
  double* Lp_s = (double*)malloc(sizeof(double) * N);
  double nrm2_s;
  double* alpha = (double*)malloc(sizeof(double) * (k + 1));

  int status = 1;
  res->nrm2_R = orc_dot(N, R, R);
  if (res->nrm2_R == 0.0) {
    for (long c = 0; c < N; ++c) x[c] = 0.0;
    res->converged = 1;
    status = 0;
    goto done;
  }
  double thr2 = (pb->tol * pb->tol) * res->nrm2_R;

  /* initialisation: r^0 = L(phi^0) - R, p^0 = P^-1(r^0), L(p^0) */
  orc_copy(N, x, phi);
  orc_apply_L(nlon, nlat, pb->mu, Tx, Ty, area, phi, r);
  for (long c = 0; c < N; ++c) r[c] = r[c] - R[c];
  double nrm2_prev = orc_dot(N, r, r);
  res->nrm2_0 = nrm2_prev;
  res->nrm2_final = nrm2_prev;
  if (nrm2_prev <= thr2) {
    orc_copy(N, phi, x);
    res->converged = 1;
    status = 0;
    goto done;
  }
  orc_solve_P(nlon, nlat, pb->mu, Tx, Ty, area, pb->precond, pb->dense_pinv, r, p[0]);
  orc_apply_L(nlon, nlat, pb->mu, Tx, Ty, area, p[0], Lp[0]);
  orc_copy(N, phi, phi_s);
  orc_copy(N, r, r_s);
  orc_copy(N, p[0], p_s);
  orc_copy(N, Lp[0], Lp_s);
  nrm2_s = nrm2_prev;

  int nu = 0;
  int64_t t = 0;
  for (;;) {
    if (t >= pb->max_steps) break;
    t = t + 1;
    res->steps = t;
    res->faults_injected += orc_inject(faults, nfaults, t, ORC_VEC_X, phi, N);
    res->faults_injected += orc_inject(faults, nfaults, t, ORC_VEC_R, r, N);
    res->faults_injected += orc_inject(faults, nfaults, t, ORC_VEC_P, p[nu], N);
    res->faults_injected += orc_inject(faults, nfaults, t, ORC_VEC_AP, Lp[nu], N);
    if (lp_trace) orc_copy(N, Lp[nu], lp_trace + (t - 1) * N);

    double beta = -orc_dot(N, r, Lp[nu]) / orc_dot(N, Lp[nu], Lp[nu]);
    for (long c = 0; c < N; ++c) {
      phin[c] = fma(beta, p[nu][c], phi[c]);
      rn[c] = fma(beta, Lp[nu][c], r[c]);
    }
    double nrm2 = orc_dot(N, rn, rn);
    if (nrm2_hist) nrm2_hist[t - 1] = nrm2;
    if (beta_hist) beta_hist[t - 1] = beta;

    if (nrm2 <= thr2) { /* exit test first */
      if (event_hist) event_hist[t - 1] = ORC_EVENT_EXIT;
      orc_copy(N, phin, x);
      res->nrm2_final = nrm2;
      res->converged = 1;
      status = 0;
      goto done;
    }
    if (pb->protect && !(nrm2 < nrm2_prev)) { /* fault: restore the backup, redo the cycle */
      if (event_hist) event_hist[t - 1] = ORC_EVENT_FAULT;
      if (res->ndetect < ORC_MAX_DETECT) res->detect_step[res->ndetect++] = t;
      res->faults_detected += 1;
      res->restarts += 1;
      orc_copy(N, phi_s, phi);
      orc_copy(N, r_s, r);
      orc_copy(N, p_s, p[0]);
      orc_copy(N, Lp_s, Lp[0]);
      nrm2_prev = nrm2_s;
      nu = 0;
      continue;
    }
    if (event_hist) event_hist[t - 1] = ORC_EVENT_ACCEPT;
    if (pb->protect && nu == 0) { /* first step of the cycle passed: ^* <- ^0 */
      orc_copy(N, phi, phi_s);
      orc_copy(N, r, r_s);
      orc_copy(N, p[0], p_s);
      orc_copy(N, Lp[0], Lp_s);
      nrm2_s = nrm2_prev;
    }
    nrm2_prev = nrm2;
    res->nrm2_final = nrm2;
    { double* tmp = phi; phi = phin; phin = tmp; }
    { double* tmp = r; r = rn; rn = tmp; }

    orc_solve_P(nlon, nlat, pb->mu, Tx, Ty, area, pb->precond, pb->dense_pinv, r, e);
    res->faults_injected += orc_inject(faults, nfaults, t, ORC_VEC_E, e, N);
    res->loss_events += orc_data_loss(losses, nlosses, t, e, N);
    orc_apply_L(nlon, nlat, pb->mu, Tx, Ty, area, e, Le);
    for (int l = 0; l <= nu; ++l) alpha[l] = -orc_dot(N, Le, Lp[l]) / orc_dot(N, Lp[l], Lp[l]);
    for (long c = 0; c < N; ++c) {
      double pa = e[c], la = Le[c];
      for (int l = 0; l <= nu; ++l) {
        pa = fma(alpha[l], p[l][c], pa);
        la = fma(alpha[l], Lp[l][c], la);
      }
      p[nu + 1][c] = pa;
      Lp[nu + 1][c] = la;
    }
    nu = nu + 1;
    if (nu == k) { /* cycle end: ^0 <- ^k */
      double* tp = p[0]; p[0] = p[k]; p[k] = tp;
      double* tl = Lp[0]; Lp[0] = Lp[k]; Lp[k] = tl;
      nu = 0;
      res->cycles += 1;
    }
  }
  orc_copy(N, phi, x); /* max_steps ran out: return the current iterate */

done:
  if (res->nrm2_R != 0.0) {
    orc_apply_L(nlon, nlat, pb->mu, Tx, Ty, area, x, e);
    for (long c = 0; c < N; ++c) e[c] = e[c] - R[c];
    res->res_true = sqrt(orc_dot(N, e, e));
  }
  free(Tx); free(Ty); free(area); free(phi); free(r); free(phin); free(rn); free(e); free(Le);
  for (int l = 0; l <= k; ++l) { free(p[l]); free(Lp[l]); }
  free(p); free(Lp); free(phi_s); free(r_s); free(p_s); free(Lp_s); free(alpha);
  return status;
}
