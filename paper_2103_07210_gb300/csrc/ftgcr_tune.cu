// Tile autotuner of libftgcr: picks, by timing, the row-band count and the
// round layout (one-pass, split or streamed rounds) of a solve shape, for a given number
// of solves of that shape sharing one persistent launch.
//
// It is a client of the public C ABI (ftgcr_create, ftgcr_solve_batch,
// ftgcr_stats, ftgcr_apply_operator, ftgcr_destroy): every candidate is a
// real handle.  A candidate whose rows do not fit on chip is refused by
// ftgcr_create and skipped.  The problem timed is the caller's operator, with
// a smooth manufactured right-hand side R = L(u) and x0 = 0; each candidate
// runs one warm launch and the best of three timed ones (CUDA events on the
// tuner's own stream).  Results are cached per (grid shape, precision,
// preconditioner, flags, k, tol, concurrency) for the life of the process.
// The paper has no counterpart: it runs one problem per MPI decomposition.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "../../include/ftgcr.h"

namespace {

// u_{j,i} = cos(theta_j) sin(3 lambda_i + theta_j): smooth, zero mean in
// longitude, so R = L(u) is a consistent right-hand side for every mu >= 0.
__global__ void k_tune_pattern(int nlon, int nlat, double* u) {
  const long long N = (long long)nlon * nlat;
  const double pi = 3.14159265358979323846;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < N; g += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(g / nlon), i = (int)(g - (long long)j * nlon);
    const double lam = 2.0 * pi * (i + 0.5) / nlon, th = -0.5 * pi + pi * (j + 0.5) / nlat;
    u[g] = cos(th) * sin(3.0 * lam + th);
  }
}

using Key = std::tuple<int, int, int, int, int, int, double, int, double, int, int, long long>;

std::mutex g_mu;
std::map<Key, ftgcr_tuning_t>& cache() {
  static std::map<Key, ftgcr_tuning_t> c;
  return c;
}

struct Scratch {
  double* buf = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<ftgcr_handle*> hs;
  ~Scratch() {
    for (ftgcr_handle* h : hs)
      if (h) ftgcr_destroy(h);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (buf) cudaFree(buf);
  }
  void release() {
    for (ftgcr_handle* h : hs)
      if (h) ftgcr_destroy(h);
    hs.clear();
  }
};

#define TK(x)                                 \
  do {                                        \
    if ((x) != cudaSuccess) {                 \
      cudaGetLastError();                     \
      return FTGCR_ERR_CUDA;                  \
    }                                         \
  } while (0)

// Time one candidate layout: create `n` handles, solve them together, best of
// three launches.  Returns FTGCR_ERR_ARG if the layout does not fit.
int time_candidate(const ftgcr_grid& g, const ftgcr_coeffs* coeffs, int32_t k, double tol, int n, Scratch& sc,
                   const double* rhs, double* const* xs, size_t N, double* ms, int* tiles, int* split) {
  sc.release();
  for (int q = 0; q < n; ++q) {
    ftgcr_handle* h = nullptr;
    const int rc = ftgcr_create(&g, coeffs, k, tol, &h);
    if (rc) return rc;
    sc.hs.push_back(h);
  }
  std::vector<const double*> rs(n, rhs);
  double best = 1e300;
  for (int rep = 0; rep < 4; ++rep) {
    for (int q = 0; q < n; ++q) TK(cudaMemsetAsync(xs[q], 0, sizeof(double) * N, sc.st));
    TK(cudaEventRecord(sc.e0, sc.st));
    const int rc = ftgcr_solve_batch(sc.hs.data(), rs.data(), xs, nullptr, n, sc.st);
    if (rc) return rc;
    TK(cudaEventRecord(sc.e1, sc.st));
    TK(cudaEventSynchronize(sc.e1));
    float t = 0.f;
    TK(cudaEventElapsedTime(&t, sc.e0, sc.e1));
    if (rep > 0) best = std::min(best, (double)t);
  }
  ftgcr_stats_t s;
  if (ftgcr_stats(sc.hs[0], &s) < 0) return FTGCR_ERR_CUDA;
  if (!s.converged) return FTGCR_NOT_CONVERGED;
  *ms = best;
  *tiles = s.tiles;
  *split = s.split_rounds;
  return FTGCR_OK;
}

}  // namespace

extern "C" int ftgcr_tune(const ftgcr_grid* grid, const ftgcr_coeffs* coeffs, int32_t k, double tol,
                          int32_t concurrency, ftgcr_tuning_t* out) {
  if (!grid || !coeffs || !coeffs->D || !out || concurrency < 1 || concurrency > FTGCR_TUNE_MAX_CONCURRENCY)
    return FTGCR_ERR_ARG;
  if (grid->tiles != 0) return FTGCR_ERR_ARG;  // the tuner chooses the bands
  if (grid->flags & (FTGCR_FLAG_SPLIT_ROUNDS | FTGCR_FLAG_FUSED_ROUNDS | FTGCR_FLAG_STREAMED_ROUNDS))
    return FTGCR_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FTGCR_ERR_CUDA;
  }
  const Key key{dev, grid->nlon, grid->nlat, grid->precision, grid->precond, grid->flags, grid->mu, k, tol,
                concurrency, grid->max_outer, (long long)grid->max_steps};
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = cache().find(key);
    if (it != cache().end()) {
      *out = it->second;
      out->cached = 1;
      return FTGCR_OK;
    }
  }
  const size_t N = (size_t)grid->nlon * grid->nlat;
  Scratch sc;
  TK(cudaStreamCreateWithFlags(&sc.st, cudaStreamNonBlocking));
  TK(cudaEventCreate(&sc.e0));
  TK(cudaEventCreate(&sc.e1));
  // the default layout: its handle also builds the right-hand side
  ftgcr_grid g = *grid;
  ftgcr_handle* h0 = nullptr;
  int rc = ftgcr_create(&g, coeffs, k, tol, &h0);
  if (rc) return rc;
  sc.hs.push_back(h0);
  TK(cudaMalloc(&sc.buf, sizeof(double) * N * (2 + (size_t)concurrency)));
  double* u = sc.buf;
  double* rhs = sc.buf + N;
  std::vector<double*> xs(concurrency);
  for (int q = 0; q < concurrency; ++q) xs[q] = sc.buf + N * (2 + (size_t)q);
  k_tune_pattern<<<256, 256, 0, sc.st>>>(grid->nlon, grid->nlat, u);
  TK(cudaGetLastError());
  rc = ftgcr_apply_operator(h0, u, rhs, sc.st);
  if (rc) return rc;
  TK(cudaStreamSynchronize(sc.st));
  // one solve with the default layout: its statistics name the layout
  TK(cudaMemsetAsync(xs[0], 0, sizeof(double) * N, sc.st));
  rc = ftgcr_solve_async(h0, rhs, xs[0], nullptr, sc.st);
  if (rc) return rc;
  TK(cudaStreamSynchronize(sc.st));
  ftgcr_stats_t s0;
  rc = ftgcr_stats(h0, &s0);
  if (rc < 0) return rc;
  const int nt_def = s0.tiles, split_def = s0.split_rounds;

  // candidates: band heights around the default one, each in both round
  // layouts where the mixed path's line preconditioner offers two
  const int nlat = grid->nlat;
  const int h_def = (nlat + nt_def - 1) / nt_def;
  std::vector<int> heights = {1, 2, 3, 4, 6, 8, 12, 16, h_def, std::max(1, h_def / 2), h_def + 1, 2 * h_def};
  std::vector<int> nts = {nt_def};
  for (int h : heights) {
    if (h < 1 || h > nlat) continue;
    const int nt = (nlat + h - 1) / h;
    if (std::find(nts.begin(), nts.end(), nt) == nts.end()) nts.push_back(nt);
  }
  std::vector<int> layouts = {0};
  if (grid->precision == FTGCR_MIXED && grid->precond == FTGCR_PRECOND_LINE) {
    layouts = {FTGCR_FLAG_FUSED_ROUNDS, FTGCR_FLAG_SPLIT_ROUNDS};
    // streamed step rounds: rows of at least one 1024-column chunk
    if (grid->nlon >= 1024) layouts.push_back(FTGCR_FLAG_STREAMED_ROUNDS);
  }
  ftgcr_tuning_t best{};
  best.ms = 1e300;
  int tried = 0;
  double ms_def = -1.0;
  for (int nt : nts)
    for (int lay : layouts) {
      g = *grid;
      g.tiles = nt;
      g.flags = grid->flags | lay;
      double ms = 0.0;
      int tiles = 0, split = 0;
      rc = time_candidate(g, coeffs, k, tol, concurrency, sc, rhs, xs.data(), N, &ms, &tiles, &split);
      if (rc == FTGCR_ERR_ARG || rc == FTGCR_ERR_OOM || rc == FTGCR_NOT_CONVERGED) {
        cudaGetLastError();
        continue;  // does not fit on chip or in memory, or did not converge
      }
      if (rc) return rc;
      ++tried;
      if (tiles == nt_def && split == split_def) ms_def = ms;
      if (ms < best.ms) {
        best.ms = ms;
        best.tiles = tiles;
        best.flags = split == 2 ? FTGCR_FLAG_STREAMED_ROUNDS
                                : (split ? FTGCR_FLAG_SPLIT_ROUNDS : (lay ? FTGCR_FLAG_FUSED_ROUNDS : 0));
      }
    }
  sc.release();
  if (!tried) return FTGCR_ERR_ARG;
  best.candidates = tried;
  best.default_tiles = nt_def;
  best.default_ms = ms_def;
  best.cached = 0;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    cache()[key] = best;
  }
  *out = best;
  return FTGCR_OK;
}
