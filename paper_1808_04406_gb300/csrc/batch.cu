// Batched sweep: many independent periodic D2Q9 CM-MRT runs of different sizes
// advance together, one kernel launch per time step for the whole batch.
//
// Every run keeps its own AA-layout slice of one population buffer (planes of
// N_r = nx_r * ny_r values, each run's slice aligned to 64 elements).  A tile
// list in the workspace covers every run: a tile is `rows` rows of one run and
// `threads` consecutive work units: node pairs in packed FP32x2 (even nx) or
// single nodes (odd nx, FP64).  Each block walks the tile list with
// a grid stride; there is no waiting between blocks inside a step, the launch
// boundary is the step barrier.  A run whose nodes went unphysical is flagged in
// its status word and skipped from then on.  The tile shape is chosen by
// lbm_batch_autotune; lbm_batch_use_graph replays a captured two-step CUDA graph.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "sweep_body.cuh"

namespace lbm {
namespace {

struct BRun {
  int64_t off;  // element offset of the run's slice
  int nx, ny;
  double om[5];  // rates of orders 0..4
  int pair;     // 1: node pairs (nx even, 16/32-bit storage); 0: single nodes
};

struct BTile {
  int run, y0, x0;  // x0 in pairs (pair runs) or nodes
};

constexpr int kMaxTileThreads = 256;

template <int S, bool ODD>
__global__ void __launch_bounds__(kMaxTileThreads)
    batch_sweep_kernel(typename tp::Store<S>::type* __restrict__ f, const BRun* __restrict__ runs,
                       const BTile* __restrict__ tiles, int ntiles, int rows, int* __restrict__ status) {
  using T = typename tp::Store<S>::calc;
  BTile next = blockIdx.x < ntiles ? tiles[blockIdx.x] : BTile{0, 0, 0};
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const BTile tl = next;  // the next tile's descriptor is fetched before this tile's work
    if (t + (int)gridDim.x < ntiles) next = tiles[t + gridDim.x];
    const BRun R = runs[tl.run];
    if (status[tl.run]) continue;  // the whole block skips a diverged run
    const tp::Grid g{R.nx, R.ny, 1, (int64_t)R.nx * R.ny};
    typename tp::Store<S>::type* fr = f + R.off;
    const int y1 = min(tl.y0 + rows, R.ny);
    bool ok = true;
    if constexpr (S != LBM_F64) {
      if (R.pair) {
        f2 om[5];
#pragma unroll
        for (int n = 0; n < 5; ++n) om[n] = cst<f2>(R.om[n]);
        const int xp = tl.x0 + threadIdx.x;
        if (xp < (R.nx >> 1)) {
          // rows of the tile in a pipeline: row y + 1's loads go out before row y's collision
          f2 cur[9], nxt[9];
          tp::pair_load<2, S, ODD>(fr, g, tp::PairAddr<2, ODD>(g, xp, tl.y0, 0), cur);
          for (int y = tl.y0; y < y1; ++y) {
            if (y + 1 < y1) tp::pair_load<2, S, ODD>(fr, g, tp::PairAddr<2, ODD>(g, xp, y + 1, 0), nxt);
            ok = tp::collide<f2, 2>(cur, om) && ok;
            tp::pair_store<2, S, ODD>(fr, g, tp::PairAddr<2, ODD>(g, xp, y, 0), cur);
#pragma unroll
            for (int j = 0; j < 9; ++j) cur[j] = nxt[j];
          }
        }
        if (!ok) atomicOr(&status[tl.run], 1);
        continue;
      }
    }
    T om[5];
#pragma unroll
    for (int n = 0; n < 5; ++n) om[n] = (T)R.om[n];
    const int x = tl.x0 + threadIdx.x;
    if (x < R.nx) {
      T cur[9], nxt[9];
      tp::node_load<2, S, ODD>(fr, g, tp::NodeAddr<2, ODD>(g, x, tl.y0, 0), cur);
      for (int y = tl.y0; y < y1; ++y) {
        if (y + 1 < y1) tp::node_load<2, S, ODD>(fr, g, tp::NodeAddr<2, ODD>(g, x, y + 1, 0), nxt);
        ok = tp::collide<T, 2>(cur, om) && ok;
        tp::node_store<2, S, ODD>(fr, g, tp::NodeAddr<2, ODD>(g, x, y, 0), cur);
#pragma unroll
        for (int j = 0; j < 9; ++j) cur[j] = nxt[j];
      }
    }
    if (!ok) atomicOr(&status[tl.run], 1);
  }
}

constexpr size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr int64_t round64(int64_t n) { return (n + 63) & ~(int64_t)63; }

struct Layout {
  std::vector<int64_t> off;  // per-run element offsets
  int64_t elems = 0;
  int64_t max_n = 0;
  int64_t max_tiles = 0;
  size_t status = 0, runs = 0, tiles = 0, results = 0, sub = 0, total = 0;
};

// 0: one node per thread (FP64); 1: node pairs (even nx); 2: node pairs plus one
// single node per row (odd nx)
// 1: node pairs in packed FP32x2 (even nx, 16/32-bit storage); 0: one node per thread.
// (Pairs at odd alignment for odd nx were measured slower on D2Q9: the alignment
// and wrap arithmetic outweighs the packed collision, 80 vs 87 GLUPS.)
int pair_run(int storage, int64_t nx) { return storage != LBM_F64 && nx % 2 == 0 ? 1 : 0; }

// work units (threads) per row
int64_t row_units(int storage, int64_t nx) { return pair_run(storage, nx) ? nx / 2 : nx; }

int64_t tiles_for(int storage, const std::vector<int64_t>& nx, const std::vector<int64_t>& ny, int threads,
                  int rows) {
  int64_t t = 0;
  for (size_t r = 0; r < nx.size(); ++r) {
    const int64_t units = row_units(storage, nx[r]);
    t += ((units + threads - 1) / threads) * ((ny[r] + rows - 1) / rows);
  }
  return t;
}

const int kThreadChoices[3] = {64, 128, 256};
const int kRowChoices[5] = {1, 2, 4, 8, 16};

int make_layout(int lattice, int n_runs, const int64_t* dims, int storage, Layout* L) {
  if (lattice != LBM_D2Q9) return set_error(LBM_EINVAL, "batched runs support the D2Q9 lattice only");
  if (n_runs < 1 || !dims) return set_error(LBM_EINVAL, "need n_runs >= 1 and dims");
  const size_t esz = storage_elem_bytes(storage);
  if (!esz) return set_error(LBM_EINVAL, "unknown storage %d", storage);
  std::vector<int64_t> nx(n_runs), ny(n_runs);
  L->off.assign(n_runs, 0);
  int64_t e = 0;
  for (int r = 0; r < n_runs; ++r) {
    nx[r] = dims[3 * r];
    ny[r] = dims[3 * r + 1];
    if (nx[r] < 1 || ny[r] < 1 || ny[r] > 65535 || dims[3 * r + 2] != 1)
      return set_error(LBM_EINVAL, "run %d: dims must be nx >= 1, 1 <= ny <= 65535, nz = 1", r);
    if ((double)nx[r] * (double)ny[r] >= 2147483648.0) return set_error(LBM_EINVAL, "run %d too large", r);
    L->off[r] = e;
    e += round64(9 * nx[r] * ny[r]);
    if (nx[r] * ny[r] > L->max_n) L->max_n = nx[r] * ny[r];
  }
  L->elems = e;
  L->max_tiles = 0;
  for (int t : kThreadChoices)
    for (int rw : kRowChoices) {
      const int64_t n = tiles_for(storage, nx, ny, t, rw);
      if (n > L->max_tiles) L->max_tiles = n;
    }
  if (L->max_tiles >= (int64_t)1 << 31) return set_error(LBM_EINVAL, "too many tiles");
  // workspace: status | run table | tiles | per-run totals | one single-run workspace
  L->status = 0;
  L->runs = L->status + round256((size_t)n_runs * sizeof(int));
  L->tiles = L->runs + round256((size_t)n_runs * sizeof(BRun));
  L->results = L->tiles + round256((size_t)L->max_tiles * sizeof(BTile));
  L->sub = L->results + round256((size_t)n_runs * 8 * sizeof(double));
  const size_t staging = std::min(kStagingMax, round256((size_t)L->max_n * 9 * sizeof(double)));
  L->total = L->sub + kWsStaging + staging;
  return LBM_OK;
}

}  // namespace

struct Batch {
  int lattice, storage, n_runs;
  std::vector<int64_t> nx, ny;
  std::vector<Rates> rates;
  Layout L;
  void* pop;
  unsigned char* work;
  cudaStream_t stream;
  int64_t step;
  int threads, rows, ntiles;
  int grid_blocks;
  bool use_graph;
  cudaGraphExec_t graph;
  int graph_parity;
  std::vector<Sim> sims;  // per-run views for fields / populations / totals

  int* status() { return reinterpret_cast<int*>(work + L.status); }
  BRun* runs_dev() { return reinterpret_cast<BRun*>(work + L.runs); }
  BTile* tiles_dev() { return reinterpret_cast<BTile*>(work + L.tiles); }
  double* results() { return reinterpret_cast<double*>(work + L.results); }
};

namespace {

int upload_tiles(Batch* b, int threads, int rows) {
  std::vector<BTile> tiles;
  tiles.reserve((size_t)tiles_for(b->storage, b->nx, b->ny, threads, rows));
  for (int r = 0; r < b->n_runs; ++r) {
    const int64_t units = row_units(b->storage, b->nx[r]);
    for (int64_t y0 = 0; y0 < b->ny[r]; y0 += rows)
      for (int64_t x0 = 0; x0 < units; x0 += threads) tiles.push_back(BTile{r, (int)y0, (int)x0});
  }
  int rc = cuda_check(cudaMemcpyAsync(b->tiles_dev(), tiles.data(), tiles.size() * sizeof(BTile),
                                      cudaMemcpyHostToDevice, b->stream),
                      "upload tiles");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(b->stream), "stream synchronize");
  if (rc) return rc;
  b->threads = threads;
  b->rows = rows;
  b->ntiles = (int)tiles.size();
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per_sm = 2048 / threads;  // resident threads per SM bound the useful grid
  const int64_t g = (int64_t)(sms > 0 ? sms : 152) * per_sm;
  b->grid_blocks = (int)(b->ntiles < g ? b->ntiles : g);
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return LBM_OK;
}

template <int S>
cudaError_t launch_batch_t(Batch* b, int odd) {
  using E = typename tp::Store<S>::type;
  E* f = static_cast<E*>(b->pop);
  if (b->ntiles == 0) return cudaSuccess;
  if (odd)
    batch_sweep_kernel<S, true><<<b->grid_blocks, b->threads, 0, b->stream>>>(f, b->runs_dev(), b->tiles_dev(),
                                                                               b->ntiles, b->rows, b->status());
  else
    batch_sweep_kernel<S, false><<<b->grid_blocks, b->threads, 0, b->stream>>>(f, b->runs_dev(), b->tiles_dev(),
                                                                                b->ntiles, b->rows, b->status());
  return cudaGetLastError();
}

cudaError_t launch_batch(Batch* b, int odd) {
  switch (b->storage) {
    case LBM_F64: return launch_batch_t<LBM_F64>(b, odd);
    case LBM_F32: return launch_batch_t<LBM_F32>(b, odd);
    case LBM_F16: return launch_batch_t<LBM_F16>(b, odd);
    case LBM_BF16: return launch_batch_t<LBM_BF16>(b, odd);
  }
  return cudaErrorInvalidValue;
}

Batch* as_batch(lbm_batch_handle h) { return reinterpret_cast<Batch*>(h); }

int check_batch(Batch* b) { return b ? LBM_OK : set_error(LBM_EINVAL, "NULL batch handle"); }

int check_run(Batch* b, int run) {
  if (int rc = check_batch(b)) return rc;
  if (run < 0 || run >= b->n_runs) return set_error(LBM_EINVAL, "run %d out of range", run);
  b->sims[run].step = b->step;  // the run's AA parity is the batch's
  b->sims[run].stream = b->stream;
  return LBM_OK;
}

// Tile-shape cache: lines "key threads rows" in the file named by LBM_AUTOTUNE_CACHE.
std::string cache_key(const Batch* b) {
  int64_t nodes = 0;
  for (int r = 0; r < b->n_runs; ++r) nodes += b->nx[r] * b->ny[r];
  char buf[128];
  snprintf(buf, sizeof(buf), "batch-d2q9-s%d-r%d-n%lld", b->storage, b->n_runs, (long long)nodes);
  return buf;
}

bool cache_lookup(const std::string& key, int* threads, int* rows) {
  const char* path = getenv("LBM_AUTOTUNE_CACHE");
  if (!path) return false;
  FILE* fp = fopen(path, "r");
  if (!fp) return false;
  char k[128];
  int t = 0, r = 0;
  bool found = false;
  while (fscanf(fp, "%127s %d %d", k, &t, &r) == 3)
    if (key == k) {
      *threads = t;
      *rows = r;
      found = true;
    }
  fclose(fp);
  return found;
}

void cache_store(const std::string& key, int threads, int rows) {
  const char* path = getenv("LBM_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* fp = fopen(path, "a");
  if (!fp) return;
  fprintf(fp, "%s %d %d\n", key.c_str(), threads, rows);
  fclose(fp);
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

int lbm_batch_query_bytes(int lattice, int n_runs, const int64_t* dims, int storage, size_t* pop_bytes,
                          size_t* work_bytes) {
  Layout L;
  if (int rc = make_layout(lattice, n_runs, dims, storage, &L)) return rc;
  if (!pop_bytes || !work_bytes) return set_error(LBM_EINVAL, "NULL output pointer");
  *pop_bytes = round256((size_t)L.elems * storage_elem_bytes(storage));
  *work_bytes = L.total;
  return LBM_OK;
}

int lbm_batch_create(int lattice, int n_runs, const int64_t* dims, const double* tau_per_order, int n_tau,
                     int storage, void* pop, size_t pop_bytes, void* work, size_t work_bytes,
                     lbm_batch_handle* out) {
  if (!out) return set_error(LBM_EINVAL, "NULL output handle pointer");
  *out = nullptr;
  Layout L;
  if (int rc = make_layout(lattice, n_runs, dims, storage, &L)) return rc;
  const size_t need_pop = round256((size_t)L.elems * storage_elem_bytes(storage));
  if (!pop || !work) return set_error(LBM_EINVAL, "NULL population or workspace buffer");
  if (pop_bytes < need_pop || work_bytes < L.total)
    return set_error(LBM_ESIZE, "buffers too small: need %zu + %zu bytes", need_pop, L.total);
  if (((uintptr_t)pop & 255) || ((uintptr_t)work & 255))
    return set_error(LBM_EINVAL, "population and workspace buffers must be 256-byte aligned");
  if (n_tau < 1 || !tau_per_order) return set_error(LBM_EINVAL, "need n_tau >= 1 times per run");
  Batch* b = new (std::nothrow) Batch();
  if (!b) return set_error(LBM_EINVAL, "host allocation failed");
  b->lattice = lattice;
  b->storage = storage;
  b->n_runs = n_runs;
  b->L = L;
  b->pop = pop;
  b->work = static_cast<unsigned char*>(work);
  b->stream = nullptr;
  b->step = 0;
  b->use_graph = false;
  b->graph = nullptr;
  b->graph_parity = 0;
  b->nx.resize(n_runs);
  b->ny.resize(n_runs);
  b->sims.resize(n_runs);
  std::vector<BRun> runs(n_runs);
  const size_t esz = storage_elem_bytes(storage);
  for (int r = 0; r < n_runs; ++r) {
    b->nx[r] = dims[3 * r];
    b->ny[r] = dims[3 * r + 1];
    BRun& R = runs[r];
    R.off = L.off[r];
    R.nx = (int)b->nx[r];
    R.ny = (int)b->ny[r];
    R.pair = pair_run(storage, b->nx[r]);
    for (int n = 0; n < 5; ++n) R.om[n] = 0.0;
    for (int n = 2; n <= 4; ++n) {
      const double t = (n - 2 < n_tau) ? tau_per_order[(size_t)r * n_tau + (n - 2)] : 1.0;
      if (!(t > 0.5) || !(t < 1e30)) {
        delete b;
        return set_error(LBM_EINVAL, "run %d: tau of order %d must exceed 1/2", r, n);
      }
      R.om[n] = 1.0 / t;
    }
    // per-run single-simulation view over the shared sub-workspace
    Sim& s = b->sims[r];
    s = Sim();
    s.lattice = LBM_D2Q9;
    s.D = 2;
    s.Q = 9;
    s.storage = storage;
    s.flags = 0;
    s.theta_ref = 1.0;
    s.nx = b->nx[r];
    s.ny = b->ny[r];
    s.nz = 1;
    s.N = s.nx * s.ny;
    for (int n = 2; n <= 4; ++n) s.rates.w[n] = R.om[n];
    s.pop = static_cast<unsigned char*>(pop) + (size_t)R.off * esz;
    s.pop_bytes = (size_t)9 * s.N * esz;
    s.work = b->work + L.sub;
    s.work_bytes = work_bytes - L.sub;
    s.staging_bytes = s.work_bytes - kWsStaging;
    s.stream = nullptr;
    s.step = 0;
  }
  int rc = cuda_check(cudaMemcpy(b->runs_dev(), runs.data(), runs.size() * sizeof(BRun), cudaMemcpyHostToDevice),
                      "upload run table");
  if (!rc) rc = cuda_check(cudaMemset(b->status(), 0, (size_t)n_runs * sizeof(int)), "clear status");
  if (!rc) rc = cuda_check(cudaMemset(b->work + L.sub, 0, 256), "clear sub-workspace status");
  if (!rc) rc = upload_tiles(b, 128, 1);
  if (rc) {
    delete b;
    return rc;
  }
  *out = reinterpret_cast<lbm_batch_handle>(b);
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch_handle h) {
  Batch* b = as_batch(h);
  if (b && b->graph) cudaGraphExecDestroy(b->graph);
  delete b;
}

int lbm_batch_set_stream(lbm_batch_handle h, void* stream) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  b->stream = static_cast<cudaStream_t>(stream);
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return LBM_OK;
}

int lbm_batch_init_run(lbm_batch_handle h, int run, const void* rho, const void* u, int dtype, int on_device) {
  Batch* b = as_batch(h);
  if (int rc = check_run(b, run)) return rc;
  if (b->step != 0) return set_error(LBM_EINVAL, "runs are initialised before the batch takes its first step");
  int rc = lbm_init_fields(reinterpret_cast<lbm_handle>(&b->sims[run]), rho, u, nullptr, dtype, on_device);
  if (!rc) rc = cuda_check(cudaMemsetAsync(b->status() + run, 0, sizeof(int), b->stream), "clear run status");
  return rc;
}

int lbm_batch_step(lbm_batch_handle h, int64_t n) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  if (n < 0) return set_error(LBM_EINVAL, "negative step count");
  int64_t k = 0;
  if (b->use_graph && n >= 2 && !b->stream)
    return set_error(LBM_EINVAL, "CUDA graphs need a non-default stream (lbm_batch_set_stream)");
  if (b->use_graph && n >= 2) {
    if (b->graph && b->graph_parity != (int)(b->step & 1)) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    if (!b->graph) {  // capture two consecutive steps from the current parity
      cudaGraph_t g = nullptr;
      int rc = cuda_check(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal), "begin capture");
      if (rc) return rc;
      cudaError_t e1 = launch_batch(b, (int)(b->step & 1));
      cudaError_t e2 = launch_batch(b, (int)((b->step + 1) & 1));
      rc = cuda_check(cudaStreamEndCapture(b->stream, &g), "end capture");
      if (!rc) rc = cuda_check(e1 != cudaSuccess ? e1 : e2, "captured sweep");
      if (!rc) rc = cuda_check(cudaGraphInstantiate(&b->graph, g, 0), "instantiate graph");
      if (g) cudaGraphDestroy(g);
      if (rc) return rc;
      b->graph_parity = (int)(b->step & 1);
    }
    for (; k + 2 <= n; k += 2) {
      int rc = cuda_check(cudaGraphLaunch(b->graph, b->stream), "graph launch");
      if (rc) return rc;
      b->step += 2;
    }
  }
  for (; k < n; ++k) {
    int rc = cuda_check(launch_batch(b, (int)(b->step & 1)), "batched sweep");
    if (rc) return rc;
    ++b->step;
  }
  return LBM_OK;
}

int lbm_batch_use_graph(lbm_batch_handle h, int enable) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  b->use_graph = enable != 0;
  return LBM_OK;
}

int lbm_batch_set_tiles(lbm_batch_handle h, int threads, int rows) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  bool okt = false, okr = false;
  for (int t : kThreadChoices) okt = okt || t == threads;
  for (int r : kRowChoices) okr = okr || r == rows;
  if (!okt || !okr) return set_error(LBM_EINVAL, "threads must be 64/128/256 and rows 1/2/4");
  return upload_tiles(b, threads, rows);
}

int lbm_batch_autotune(lbm_batch_handle h, int steps_per_trial, int* threads, int* rows) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  if (b->step != 0) return set_error(LBM_EINVAL, "autotune runs before the first step");
  if (steps_per_trial < 2) return set_error(LBM_EINVAL, "steps_per_trial must be >= 2");
  const std::string key = cache_key(b);
  int bt = 0, br = 0;
  if (!cache_lookup(key, &bt, &br)) {
    // time every tile shape on the rest state (zero offsets), a fixed point of the step
    int rc = cuda_check(cudaMemsetAsync(b->pop, 0, (size_t)b->L.elems * storage_elem_bytes(b->storage), b->stream),
                        "rest state");
    if (rc) return rc;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int t : kThreadChoices)
      for (int r : kRowChoices) {
        rc = upload_tiles(b, t, r);
        for (int k = 0; k < 2 && !rc; ++k) rc = cuda_check(launch_batch(b, k & 1), "warm-up sweep");
        if (!rc) rc = cuda_check(cudaEventRecord(e0, b->stream), "event");
        for (int k = 0; k < steps_per_trial && !rc; ++k) rc = cuda_check(launch_batch(b, k & 1), "timed sweep");
        if (!rc) rc = cuda_check(cudaEventRecord(e1, b->stream), "event");
        if (!rc) rc = cuda_check(cudaEventSynchronize(e1), "event sync");
        float ms = 0.0f;
        if (!rc) cudaEventElapsedTime(&ms, e0, e1);
        if (rc) break;
        if (ms < best) {
          best = ms;
          bt = t;
          br = r;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    // the trials took an even number of steps from the rest state: still at rest, parity even
    rc = cuda_check(cudaMemsetAsync(b->pop, 0, (size_t)b->L.elems * storage_elem_bytes(b->storage), b->stream),
                    "rest state");
    if (rc) return rc;
    cache_store(key, bt, br);
  }
  if (threads) *threads = bt;
  if (rows) *rows = br;
  return upload_tiles(b, bt, br);
}

int lbm_batch_status(lbm_batch_handle h, int* flags) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  if (!flags) return set_error(LBM_EINVAL, "NULL output pointer");
  std::vector<int> st(b->n_runs);
  int rc = cuda_check(cudaMemcpyAsync(st.data(), b->status(), st.size() * sizeof(int), cudaMemcpyDeviceToHost,
                                      b->stream),
                      "status readback");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(b->stream), "stream synchronize");
  if (rc) return rc;
  for (int r = 0; r < b->n_runs; ++r) flags[r] = st[r] ? LBM_EDIVERGED : LBM_OK;
  return LBM_OK;
}

int lbm_batch_reduce(lbm_batch_handle h, double* out) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  if (!out) return set_error(LBM_EINVAL, "NULL output pointer");
  int rc = LBM_OK;
  for (int r = 0; r < b->n_runs && !rc; ++r) {
    check_run(b, r);
    Sim& s = b->sims[r];
    rc = cuda_check(launch_reduce_into(&s, partials_buf(&s), kRedBlocks, b->results() + 8 * r), "run totals");
  }
  std::vector<double> tmp((size_t)8 * b->n_runs);
  if (!rc)
    rc = cuda_check(cudaMemcpyAsync(tmp.data(), b->results(), tmp.size() * sizeof(double), cudaMemcpyDeviceToHost,
                                    b->stream),
                    "copy totals");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(b->stream), "stream synchronize");
  if (!rc)
    for (int r = 0; r < b->n_runs; ++r)
      for (int k = 0; k < 5; ++k) out[5 * r + k] = tmp[8 * r + k];
  return rc;
}

int lbm_batch_moments(lbm_batch_handle h, int run, void* rho, void* u, int dtype, int on_device) {
  Batch* b = as_batch(h);
  if (int rc = check_run(b, run)) return rc;
  return lbm_moments(reinterpret_cast<lbm_handle>(&b->sims[run]), rho, u, nullptr, dtype, on_device);
}

int lbm_batch_get_populations(lbm_batch_handle h, int run, double* f, int on_device) {
  Batch* b = as_batch(h);
  if (int rc = check_run(b, run)) return rc;
  return lbm_get_populations(reinterpret_cast<lbm_handle>(&b->sims[run]), f, on_device);
}

int64_t lbm_batch_step_count(lbm_batch_handle h) {
  Batch* b = as_batch(h);
  return b ? b->step : -1;
}

}  // extern "C"
