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
#include <exception>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "batch_stage.cuh"
#include "reduce.cuh"
#include "sweep_body.cuh"

namespace lbm {
// lbm_abi.cu: the device address of page-locked host memory, or nullptr.
void* pinned_device_view(const void* p);
namespace {

// How the threads of a run's tiles cover its nodes.
enum RunKind : int {
  kNode = 0,   // one node per thread (FP64 storage)
  kXPair = 1,  // x-neighbour pairs in packed FP32x2 (even nx, 16/32-bit storage)
  kYPair = 2,  // column pairs (x, y), (x, y + 1) in packed FP32x2 (odd nx, 16/32-bit storage)
};

struct BRun {
  int64_t off;  // element offset of the run's slice
  int nx, ny;
  double om[5];  // rates of orders 0..4
  int kind;      // RunKind
  uint32_t m_nx, m_half;  // division magics for nx and nx / 2 (staged sweep)
};

struct BTile {
  int run, y0, x0;  // x0 in pairs (x-pair runs) or nodes
};

constexpr int kMaxTileThreads = 256;

// A thread's node pair in a tile column, with 32-bit element indices into the
// run's slice (9 nx ny < 2^32): x-neighbour pairs (even nx) ...  The pairing
// is that of the single-grid pair sweep: (x0, x0 + 1) with x0 even in the even
// sweep; (x0, x0 + 1 mod nx) with x0 odd in the odd sweep, so that the slots
// shifted by e_x = +-1 start at an even x and only e_x = 0 needs two 1-element
// accesses.
template <int S, bool ODD>
struct XPairOps {
  using E = typename PairIO<S>::E;
  using IO = PairIO<S>;
  uint32_t nx, ny, N;
  uint32_t x0, x1;  // lane 0's and lane 1's column (odd sweep: x1 = x0 + 1 mod nx)
  __device__ __forceinline__ XPairOps(const BRun& R, int xp) {
    nx = (uint32_t)R.nx;
    ny = (uint32_t)R.ny;
    N = nx * ny;
    x0 = 2u * (uint32_t)xp + (ODD ? 1u : 0u);
    x1 = x0 + 1 == nx ? 0u : x0 + 1;
  }
  // row offsets (times nx) of y - 1, y, y + 1 (periodic)
  __device__ __forceinline__ void rows(int y, uint32_t (&r)[3]) const {
    r[1] = nx * (uint32_t)y;
    r[0] = (y == 0 ? ny - 1 : (uint32_t)y - 1) * nx;
    r[2] = ((uint32_t)y + 1 == ny ? 0u : (uint32_t)y + 1) * nx;
  }
  // start of the aligned 2-element slot of population j (not for e_x = 0 in the odd sweep)
  __device__ __forceinline__ uint32_t at(int j, const uint32_t (&r)[3]) const {
    const int dx = tp::dig(j, 0), dy = tp::dig(j, 1);
    if (!ODD) return (uint32_t)j * N + r[1] + x0;
    return (uint32_t)j * N + r[dy] + (dx == 0 ? x0 - 1 : x1);
  }
  __device__ __forceinline__ void load(const E* f, int y, RawPair (&v)[9]) const {
    uint32_t r[3];
    rows(y, r);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      if (ODD && tp::dig(j, 0) == 1) {
        const uint32_t b = (uint32_t)j * N + r[tp::dig(j, 1)];
        IO::raw11(f + b + x0, f + b + x1, v[j]);
      } else {
        IO::raw2(f + at(j, r), v[j]);
      }
    }
  }
  __device__ __forceinline__ void decode(const RawPair (&r)[9], f2 (&v)[9]) const { tp::pair_decode<2, S, ODD>(r, v); }
  __device__ __forceinline__ void store(E* f, int y, const f2 (&v)[9]) const {
    uint32_t r[3];
    rows(y, r);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      f2 val = ODD ? v[j] : v[tp::opp<2>(j)];
      if (IO::kScaled) val = val * cst<f2>(tp::iwq<2>(j));
      if (ODD && tp::dig(j, 0) == 1) {
        const uint32_t b = (uint32_t)j * N + r[tp::dig(j, 1)];
        IO::store11(f + b + x0, f + b + x1, val);
      } else {
        IO::store2(f + at(j, r), val);
      }
    }
  }
};

// ... or column pairs (x, y), (x, y + 1) (odd nx); on the last row of an odd ny
// lane 1 repeats lane 0's node (same slots, same values).
template <int S, bool ODD>
struct YPairOps {
  using E = typename PairIO<S>::E;
  using IO = PairIO<S>;
  uint32_t nx, ny, N;
  uint32_t xo[3];  // column of x + e_x (odd sweep) or x
  __device__ __forceinline__ YPairOps(const BRun& R, int x) {
    nx = (uint32_t)R.nx;
    ny = (uint32_t)R.ny;
    N = nx * ny;
    xo[1] = (uint32_t)x;
    xo[0] = x == 0 ? nx - 1 : (uint32_t)x - 1;
    xo[2] = (uint32_t)x + 1 == nx ? 0u : (uint32_t)x + 1;
  }
  // row offsets (times nx) of lane 0 (a) and lane 1 (b) for e_y = -1, 0, +1
  __device__ __forceinline__ void rows(int y, uint32_t (&a)[3], uint32_t (&b)[3]) const {
    const uint32_t y0 = (uint32_t)y, y1 = y0 + 1 < ny ? y0 + 1 : y0;
    a[1] = y0 * nx;
    b[1] = y1 * nx;
    if (ODD) {
      a[0] = (y0 == 0 ? ny - 1 : y0 - 1) * nx;
      a[2] = (y0 + 1 == ny ? 0u : y0 + 1) * nx;
      b[0] = (y1 == 0 ? ny - 1 : y1 - 1) * nx;
      b[2] = (y1 + 1 == ny ? 0u : y1 + 1) * nx;
    }
  }
  __device__ __forceinline__ uint32_t col(int j) const { return ODD ? xo[tp::dig(j, 0)] : xo[1]; }
  __device__ __forceinline__ uint32_t row(int j, const uint32_t (&r)[3]) const { return ODD ? r[tp::dig(j, 1)] : r[1]; }
  __device__ __forceinline__ void load(const E* f, int y, RawPair (&v)[9]) const {
    uint32_t a[3], b[3];
    rows(y, a, b);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      const uint32_t c = (uint32_t)j * N + col(j);
      IO::raw11(f + c + row(j, a), f + c + row(j, b), v[j]);
    }
  }
  __device__ __forceinline__ void decode(const RawPair (&r)[9], f2 (&v)[9]) const { tp::ypair_decode<S, ODD>(r, v); }
  __device__ __forceinline__ void store(E* f, int y, const f2 (&v)[9]) const {
    uint32_t a[3], b[3];
    rows(y, a, b);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
      f2 val = ODD ? v[j] : v[tp::opp<2>(j)];
      if (IO::kScaled) val = val * cst<f2>(tp::iwq<2>(j));
      const uint32_t c = (uint32_t)j * N + col(j);
      IO::store11(f + c + row(j, a), f + c + row(j, b), val);
    }
  }
};

// One thread's walk down a tile: rows y0, y0 + dy, ... < y1, with the raw loads
// of the next DEPTH rows in flight while a row is collided and stored (AA slots
// belong to exactly one node per step, so the reordering is race-free).
template <int DEPTH, class Ops>
__device__ __forceinline__ bool walk_pairs(const Ops& op, typename Ops::E* __restrict__ f, const f2 (&om)[5], int y0,
                                           int y1, int dy) {
  bool ok = true;
  RawPair ra[9], rb[9];
  f2 v[9];
  op.load(f, y0, ra);
  if (DEPTH == 2 && y0 + dy < y1) op.load(f, y0 + dy, rb);
  for (int y = y0; y < y1; y += DEPTH * dy) {
    op.decode(ra, v);
    if (y + DEPTH * dy < y1) op.load(f, y + DEPTH * dy, ra);
    ok = tp::collide<f2, 2>(v, om) && ok;
    op.store(f, y, v);
    if (DEPTH == 2 && y + dy < y1) {
      op.decode(rb, v);
      if (y + 3 * dy < y1) op.load(f, y + 3 * dy, rb);
      ok = tp::collide<f2, 2>(v, om) && ok;
      op.store(f, y + dy, v);
    }
  }
  return ok;
}

// KIND >= 0: every tile is of that kind (one launch per kind); KIND < 0: the
// kind is read from the run table per tile.  `rows` counts the rows a thread
// walks (row pairs for column-pair runs).
template <int S, bool ODD, int KIND, int DEPTH>
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
    const int kind = KIND >= 0 ? KIND : R.kind;
    bool ok = true;
    if constexpr (S != LBM_F64) {
      if (kind != kNode) {
        f2 om[5];
#pragma unroll
        for (int n = 0; n < 5; ++n) om[n] = cst<f2>(R.om[n]);
        if (kind == kXPair) {
          const int xp = tl.x0 + threadIdx.x;
          if (xp < (R.nx >> 1))
            ok = walk_pairs<DEPTH>(XPairOps<S, ODD>(R, xp), fr, om, tl.y0, min(tl.y0 + rows, R.ny), 1);
        } else {
          const int x = tl.x0 + threadIdx.x;
          if (x < R.nx) ok = walk_pairs<DEPTH>(YPairOps<S, ODD>(R, x), fr, om, tl.y0, min(tl.y0 + 2 * rows, R.ny), 2);
        }
        if (!ok) atomicOr(&status[tl.run], 1);
        continue;
      }
    }
    if constexpr (KIND < 0 || KIND == kNode) {
      T om[5];
#pragma unroll
      for (int n = 0; n < 5; ++n) om[n] = (T)R.om[n];
      const int x = tl.x0 + threadIdx.x;
      const int y1 = min(tl.y0 + rows, R.ny);
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
}

// All runs' FP64 totals in one launch: block r sums run r (threads stride over
// its nodes), per node the quantities of the single-grid reduction: rho - 1,
// rho u_d and rho |u|^2 / 2 from the offsets of the parity's AA slots, each in
// the compute type and added in FP64 in a fixed order.
template <int S>
__global__ void __launch_bounds__(kAuxThreads)
    batch_reduce_kernel(const typename tp::Store<S>::type* __restrict__ f, const BRun* __restrict__ runs, int odd,
                        double* __restrict__ out) {
  using T = typename tp::Store<S>::calc;
  const BRun R = runs[blockIdx.x];
  const int64_t N = (int64_t)R.nx * R.ny;
  const tp::Grid g{R.nx, R.ny, 1, N};
  double acc[5] = {0, 0, 0, 0, 0};
  for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
    const int y = (int)(n / R.nx), x = (int)(n - (int64_t)y * R.nx);
    T v[9];
    tp::gather<2, S>(f + R.off, g, x, y, 0, odd, v);
    T drho = 0, j[2] = {0, 0};
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      drho += v[i];
#pragma unroll
      for (int d = 0; d < 2; ++d) {
        if (tp::dig(i, d) == 2) j[d] += v[i];
        if (tp::dig(i, d) == 0) j[d] -= v[i];
      }
    }
    acc[0] += (double)drho;
    acc[1] += (double)j[0];
    acc[2] += (double)j[1];
    acc[4] += (double)(T(0.5) * (j[0] * j[0] + j[1] * j[1]) / (T(1) + drho));
  }
  block_sum<5>(acc);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < 5; ++k) out[8 * (size_t)blockIdx.x + k] = acc[k];
  }
}

// Device-visible field arrays of one run (page-locked host memory seen through
// its device address, or device memory).
struct BInitPtrs {
  const void* rho;
  const void* u;
};

// Every run to the equilibrium of its fields in one launch: blocks (., r) walk
// run r's nodes.  The same per-node arithmetic as the single-run initialisation
// (f_eq of rho - 1 and u in the compute type, encoded to the even AA slots).
template <int S, typename F>
__global__ void __launch_bounds__(kAuxThreads)
    batch_init_kernel(typename tp::Store<S>::type* __restrict__ f, const BRun* __restrict__ runs,
                      const BInitPtrs* __restrict__ ptrs) {
  using T = typename tp::Store<S>::calc;
  const int r = blockIdx.y;
  const BRun R = runs[r];
  const int64_t N = (int64_t)R.nx * R.ny;
  const F* __restrict__ rho = static_cast<const F*>(ptrs[r].rho);
  const F* __restrict__ u = static_cast<const F*>(ptrs[r].u);
  const tp::Grid g{R.nx, R.ny, 1, N};
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < N; k += (int64_t)gridDim.x * blockDim.x) {
    const int y = (int)(k / R.nx), x = (int)(k - (int64_t)y * R.nx);
    T uu[2] = {(T)u[k], (T)u[N + k]};
    const T drho = (T)((double)rho[k] - 1.0);
    T v[9];
    tp::equilibrium<T, 2>(v, drho, uu);
    tp::scatter<2, S>(f + R.off, g, x, y, 0, 0, v);
  }
}

constexpr size_t round256(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr int64_t round64(int64_t n) { return (n + 63) & ~(int64_t)63; }

struct Layout {
  std::vector<int64_t> off;  // per-run element offsets
  int64_t elems = 0;
  int64_t max_n = 0;
  int64_t max_tiles = 0;
  int64_t max_bands = 0;  // of the odd sweep's lists (the even sweep's are never longer)
  size_t status = 0, runs = 0, tiles = 0, bands = 0, bands_even = 0, results = 0, init_table = 0, sub = 0,
         total = 0;
};

// Runs the staged sweep (shape `variant`) can take: 16/32-bit storage, whole rows within one band.
bool stage_run(int storage, int variant, int64_t nx) {
  if (storage == LBM_F64) return false;
  return nx <= stg::kMaxNx && nx <= stg::capacity(variant, (int)storage_elem_bytes(storage));
}

// Bands of one staged run for the odd sweep: rows 0 and ny - 1 alone (their
// spans wrap around y), the rows between in bands of as many whole rows as fit.
// The even sweep reads and writes each node's own slots, so no span wraps: its
// bands are as many whole rows as fit from row 0 on.
std::vector<stg::Band> run_bands(int storage, int variant, int r, int64_t nx, int64_t ny, bool odd = true) {
  std::vector<stg::Band> out;
  if (!odd) {
    const int64_t br = std::max<int64_t>(1, stg::capacity(variant, (int)storage_elem_bytes(storage)) / nx);
    for (int64_t y0 = 0; y0 < ny; y0 += br) out.push_back(stg::Band{r, (int)y0, (int)std::min<int64_t>(br, ny - y0), 0});
    return out;
  }
  out.push_back(stg::Band{r, 0, 1, 0});
  if (ny == 1) return out;
  const int64_t br = std::max<int64_t>(1, stg::capacity(variant, (int)storage_elem_bytes(storage)) / nx);
  for (int64_t y0 = 1; y0 < ny - 1; y0 += br)
    out.push_back(stg::Band{r, (int)y0, (int)std::min<int64_t>(br, ny - 1 - y0), 0});
  out.push_back(stg::Band{r, (int)(ny - 1), 1, 0});
  return out;
}

// Node pairs in packed FP32x2 for 16/32-bit storage: x-neighbour pairs when nx
// is even (aligned 2-element accesses), column pairs when nx is odd (1-element
// accesses; x-pairs at odd alignment were measured slower on D2Q9, 80 vs 87
// GLUPS, the alignment and wrap arithmetic outweighing the packed collision).
int run_kind(int storage, int64_t nx) {
  if (storage == LBM_F64) return kNode;
  return nx % 2 == 0 ? kXPair : kYPair;
}

// work units (threads) per row, and rows covered by one tile of `rows`
int64_t row_units(int kind, int64_t nx) { return kind == kXPair ? nx / 2 : nx; }
int64_t tile_rows(int kind, int rows) { return kind == kYPair ? 2 * (int64_t)rows : rows; }

int64_t tiles_for(int storage, const std::vector<int64_t>& nx, const std::vector<int64_t>& ny, int threads,
                  int rows) {
  int64_t t = 0;
  for (size_t r = 0; r < nx.size(); ++r) {
    const int kind = run_kind(storage, nx[r]);
    const int64_t units = row_units(kind, nx[r]), tr = tile_rows(kind, rows);
    t += ((units + threads - 1) / threads) * ((ny[r] + tr - 1) / tr);
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
    if (9.0 * (double)nx[r] * (double)ny[r] >= 4294967296.0)
      return set_error(LBM_EINVAL, "run %d too large (9 nx ny must stay below 2^32)", r);
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
  L->max_bands = 0;
  for (int v = 0; v < stg::kVariants; ++v) {
    int64_t nb = 0;
    for (int r = 0; r < n_runs; ++r)
      if (stage_run(storage, v, nx[r])) nb += (int64_t)run_bands(storage, v, r, nx[r], ny[r]).size();
    L->max_bands = std::max(L->max_bands, nb);
  }
  L->tiles = L->runs + round256((size_t)n_runs * sizeof(BRun));
  L->bands = L->tiles + round256((size_t)L->max_tiles * sizeof(BTile));
  L->bands_even = L->bands + round256((size_t)L->max_bands * sizeof(stg::Band));
  L->results = L->bands_even + round256((size_t)L->max_bands * sizeof(stg::Band));
  L->init_table = L->results + round256((size_t)n_runs * 8 * sizeof(double));
  L->sub = L->init_table + round256((size_t)n_runs * 2 * sizeof(void*));
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
  int kind_tiles[3];  // tiles of each RunKind; the list holds x-pair, column-pair, then node tiles
  bool split;         // one launch per run kind (each specialised) instead of one for all tiles
  int depth;          // rows whose loads a thread keeps in flight (1 or 2)
  int staged;         // 0: tile sweep only; v + 1: staged sweep of shape v for the runs it can take
  int nbands, nbands_even;  // the odd and the even sweep's band lists
  int sms;
  int grid_blocks;
  bool use_graph;
  cudaGraphExec_t graph;
  int graph_parity;
  std::vector<Sim> sims;  // per-run views for fields / populations / totals

  int* status() { return reinterpret_cast<int*>(work + L.status); }
  BRun* runs_dev() { return reinterpret_cast<BRun*>(work + L.runs); }
  BTile* tiles_dev() { return reinterpret_cast<BTile*>(work + L.tiles); }
  stg::Band* bands_dev() { return reinterpret_cast<stg::Band*>(work + L.bands); }
  stg::Band* bands_even_dev() { return reinterpret_cast<stg::Band*>(work + L.bands_even); }
  double* results() { return reinterpret_cast<double*>(work + L.results); }
};

namespace {

// LBM_BATCH_EVEN_BANDS=0 gives the even sweep the odd sweep's band list, with
// the one-row edge bands (read when the band lists are built; used to compare).
bool even_bands() {
  const char* e = std::getenv("LBM_BATCH_EVEN_BANDS");
  return !(e && std::strcmp(e, "0") == 0);
}

int upload_tiles(Batch* b, int threads, int rows, bool split, int depth, int staged) {
  std::vector<BTile> tiles;
  std::vector<stg::Band> bands, bands_even;
  tiles.reserve((size_t)tiles_for(b->storage, b->nx, b->ny, threads, rows));
  const int order[3] = {kXPair, kYPair, kNode};
  for (int k : order) {
    const size_t before = tiles.size();
    for (int r = 0; r < b->n_runs; ++r) {
      if (run_kind(b->storage, b->nx[r]) != k || (staged && stage_run(b->storage, staged - 1, b->nx[r]))) continue;
      const int64_t units = row_units(k, b->nx[r]), tr = tile_rows(k, rows);
      for (int64_t y0 = 0; y0 < b->ny[r]; y0 += tr)
        for (int64_t x0 = 0; x0 < units; x0 += threads) tiles.push_back(BTile{r, (int)y0, (int)x0});
    }
    b->kind_tiles[k] = (int)(tiles.size() - before);
  }
  if (staged)
    for (int r = 0; r < b->n_runs; ++r) {
      if (!stage_run(b->storage, staged - 1, b->nx[r])) continue;
      const std::vector<stg::Band> rb = run_bands(b->storage, staged - 1, r, b->nx[r], b->ny[r]);
      bands.insert(bands.end(), rb.begin(), rb.end());
      const std::vector<stg::Band> re = run_bands(b->storage, staged - 1, r, b->nx[r], b->ny[r], !even_bands());
      bands_even.insert(bands_even.end(), re.begin(), re.end());
    }
  int rc = LBM_OK;
  if (!tiles.empty())
    rc = cuda_check(cudaMemcpyAsync(b->tiles_dev(), tiles.data(), tiles.size() * sizeof(BTile),
                                    cudaMemcpyHostToDevice, b->stream),
                    "upload tiles");
  if (!rc && !bands.empty())
    rc = cuda_check(cudaMemcpyAsync(b->bands_dev(), bands.data(), bands.size() * sizeof(stg::Band),
                                    cudaMemcpyHostToDevice, b->stream),
                    "upload bands");
  if (!rc && !bands_even.empty())
    rc = cuda_check(cudaMemcpyAsync(b->bands_even_dev(), bands_even.data(), bands_even.size() * sizeof(stg::Band),
                                    cudaMemcpyHostToDevice, b->stream),
                    "upload bands");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(b->stream), "stream synchronize");
  if (rc) return rc;
  b->threads = threads;
  b->rows = rows;
  b->split = split;
  b->depth = depth;
  b->staged = staged;
  b->ntiles = (int)tiles.size();
  b->nbands = (int)bands.size();
  b->nbands_even = (int)bands_even.size();
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (sms <= 0) sms = 152;
  const int per_sm = 2048 / threads;  // resident threads per SM bound the useful grid
  b->grid_blocks = sms * per_sm;
  b->sms = sms;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return LBM_OK;
}

template <int S, bool ODD, int KIND>
void launch_tiles(Batch* b, const BTile* tiles, int n) {
  using E = typename tp::Store<S>::type;
  if (n <= 0) return;
  const int grid = n < b->grid_blocks ? n : b->grid_blocks;
  E* f = static_cast<E*>(b->pop);
  if (b->depth == 2)
    batch_sweep_kernel<S, ODD, KIND, 2><<<grid, b->threads, 0, b->stream>>>(f, b->runs_dev(), tiles, n, b->rows,
                                                                             b->status());
  else
    batch_sweep_kernel<S, ODD, KIND, 1><<<grid, b->threads, 0, b->stream>>>(f, b->runs_dev(), tiles, n, b->rows,
                                                                             b->status());
}

template <int S, bool ODD>
void launch_parity(Batch* b) {
  if (!b->split) {
    launch_tiles<S, ODD, -1>(b, b->tiles_dev(), b->ntiles);
    return;
  }
  const BTile* t = b->tiles_dev();
  if constexpr (S != LBM_F64) {
    launch_tiles<S, ODD, kXPair>(b, t, b->kind_tiles[kXPair]);
    launch_tiles<S, ODD, kYPair>(b, t + b->kind_tiles[kXPair], b->kind_tiles[kYPair]);
  } else {
    launch_tiles<S, ODD, kNode>(b, t, b->kind_tiles[kNode]);
  }
}

template <class C, int S, bool ODD>
void launch_variant(Batch* b) {
  const int cap = b->sms * C::kMinBlocks;
  const int nb = ODD ? b->nbands : b->nbands_even;
  const int grid = nb < cap ? nb : cap;
  stg::staged_kernel<C, S, ODD, BRun><<<grid, C::kThreads, C::kSmemBytes, b->stream>>>(
      static_cast<typename PairIO<S>::E*>(b->pop), b->runs_dev(), ODD ? b->bands_dev() : b->bands_even_dev(), nb,
      b->status());
}

template <int S, bool ODD>
void launch_staged(Batch* b) {
  if constexpr (S != LBM_F64) {
    if (!b->staged || (ODD ? b->nbands : b->nbands_even) <= 0) return;
    switch (b->staged - 1) {
      case 0: launch_variant<stg::V0, S, ODD>(b); break;
      case 1: launch_variant<stg::V1, S, ODD>(b); break;
      case 2: launch_variant<stg::V2, S, ODD>(b); break;
      case 3: launch_variant<stg::V3, S, ODD>(b); break;
    }
  }
}

template <int S>
cudaError_t launch_batch_t(Batch* b, int odd) {
  if (odd) {
    launch_staged<S, true>(b);
    if (b->ntiles) launch_parity<S, true>(b);
  } else {
    launch_staged<S, false>(b);
    if (b->ntiles) launch_parity<S, false>(b);
  }
  return cudaGetLastError();
}

// Opt the staged kernels in to their dynamic shared memory.
template <class C, int S>
cudaError_t prepare_variant() {
  cudaError_t e = cudaFuncSetAttribute(stg::staged_kernel<C, S, false, BRun>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, C::kSmemBytes);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(stg::staged_kernel<C, S, true, BRun>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             C::kSmemBytes);
  return e;
}

template <int S>
cudaError_t prepare_storage() {
  cudaError_t e = prepare_variant<stg::V0, S>();
  if (e == cudaSuccess) e = prepare_variant<stg::V1, S>();
  if (e == cudaSuccess) e = prepare_variant<stg::V2, S>();
  if (e == cudaSuccess) e = prepare_variant<stg::V3, S>();
  return e;
}

int prepare_staged(int storage) {
  cudaError_t e = cudaSuccess;
  switch (storage) {
    case LBM_F32: e = prepare_storage<LBM_F32>(); break;
    case LBM_F16: e = prepare_storage<LBM_F16>(); break;
    case LBM_BF16: e = prepare_storage<LBM_BF16>(); break;
  }
  return cuda_check(e, "staged sweep shared-memory size");
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

// Launch-shape cache: lines "key threads rows split depth staged" in the file named by LBM_AUTOTUNE_CACHE.
std::string cache_key(const Batch* b) {
  int64_t nodes = 0;
  for (int r = 0; r < b->n_runs; ++r) nodes += b->nx[r] * b->ny[r];
  char buf[128];
  snprintf(buf, sizeof(buf), "batch4-d2q9-s%d-r%d-n%lld", b->storage, b->n_runs, (long long)nodes);
  return buf;
}

bool cache_lookup(const std::string& key, int* threads, int* rows, int* split, int* depth, int* staged) {
  const char* path = getenv("LBM_AUTOTUNE_CACHE");
  if (!path) return false;
  FILE* fp = fopen(path, "r");
  if (!fp) return false;
  char line[256], k[128];
  int t = 0, r = 0, sp = 0, dp = 0, sg = 0;
  bool found = false;
  while (fgets(line, sizeof(line), fp))
    if (sscanf(line, "%127s %d %d %d %d %d", k, &t, &r, &sp, &dp, &sg) == 6 && key == k) {
      *threads = t;
      *rows = r;
      *split = sp;
      *depth = dp;
      *staged = sg;
      found = true;
    }
  fclose(fp);
  return found;
}

void cache_store(const std::string& key, int threads, int rows, int split, int depth, int staged) {
  const char* path = getenv("LBM_AUTOTUNE_CACHE");
  if (!path) return;
  FILE* fp = fopen(path, "a");
  if (!fp) return;
  fprintf(fp, "%s %d %d %d %d %d\n", key.c_str(), threads, rows, split, depth, staged);
  fclose(fp);
}

template <int S>
cudaError_t launch_batch_init_t(Batch* b, const BInitPtrs* table, int dtype) {
  using E = typename tp::Store<S>::type;
  const int64_t max_n = b->L.max_n;
  const int64_t per_run = (max_n + kAuxThreads - 1) / kAuxThreads;  // blocks a run could use
  dim3 grid((unsigned)(per_run < 64 ? per_run : 64), (unsigned)b->n_runs);
  E* f = static_cast<E*>(b->pop);
  if (dtype == LBM_DTYPE_F64)
    batch_init_kernel<S, double><<<grid, kAuxThreads, 0, b->stream>>>(f, b->runs_dev(), table);
  else
    batch_init_kernel<S, float><<<grid, kAuxThreads, 0, b->stream>>>(f, b->runs_dev(), table);
  return cudaGetLastError();
}

}  // namespace
}  // namespace lbm

using namespace lbm;

// Host-side fault injection for tests: when the environment variable
// LBM_FAULT_HOST_ALLOC names `site`, the host allocation that follows is
// treated as failed (std::bad_alloc).  No device state is touched.
static void host_fault_point(const char* site) {
  const char* want = std::getenv("LBM_FAULT_HOST_ALLOC");
  if (want && std::strcmp(want, site) == 0) throw std::bad_alloc();
}

// Every int-returning entry point runs its body under host_guard: the bodies
// build host containers (tile and band lists, per-run tables, the autotuner's
// cache key), and a failed host allocation there must come back as LBM_EOOM
// instead of unwinding through the C boundary.
template <class F>
int host_guard(const char* call, F&& body) {
  try {
    return body();
  } catch (const std::bad_alloc&) {
    return set_error(LBM_EOOM, "%s: host allocation failed", call);
  } catch (const std::exception& e) {
    return set_error(LBM_EINVAL, "%s: %s", call, e.what());
  } catch (...) {
    return set_error(LBM_EINVAL, "%s: unexpected host exception", call);
  }
}

extern "C" {

static int lbm_batch_query_bytes_body(int lattice, int n_runs, const int64_t* dims, int storage, size_t* pop_bytes,
                          size_t* work_bytes) {
  Layout L;
  if (int rc = make_layout(lattice, n_runs, dims, storage, &L)) return rc;
  if (!pop_bytes || !work_bytes) return set_error(LBM_EINVAL, "NULL output pointer");
  *pop_bytes = round256((size_t)L.elems * storage_elem_bytes(storage));
  *work_bytes = L.total;
  return LBM_OK;
}

static int lbm_batch_create_body(int lattice, int n_runs, const int64_t* dims, const double* tau_per_order, int n_tau,
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
  std::unique_ptr<Batch> hold(new (std::nothrow) Batch());
  Batch* b = hold.get();
  if (!b) return set_error(LBM_EOOM, "host allocation of the batch handle failed");
  host_fault_point("lbm_batch_create");
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
    R.kind = run_kind(storage, b->nx[r]);
    R.m_nx = stg::div_magic((uint32_t)std::min<int64_t>(b->nx[r], stg::kMaxNx));
    R.m_half = stg::div_magic((uint32_t)std::max<int64_t>(1, std::min<int64_t>(b->nx[r] / 2, stg::kMaxNx)));
    for (int n = 0; n < 5; ++n) R.om[n] = 0.0;
    for (int n = 2; n <= 4; ++n) {
      const double t = (n - 2 < n_tau) ? tau_per_order[(size_t)r * n_tau + (n - 2)] : 1.0;
      if (!(t > 0.5) || !(t < 1e30)) return set_error(LBM_EINVAL, "run %d: tau of order %d must exceed 1/2", r, n);
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
  if (!rc) rc = cuda_check(cudaMemset(b->work + L.sub, 0, 512), "clear sub-workspace status and results");
  if (!rc) rc = prepare_staged(storage);
  if (!rc) rc = upload_tiles(b, 128, 1, false, 1, 1);
  if (rc) return rc;
  *out = reinterpret_cast<lbm_batch_handle>(hold.release());
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch_handle h) {
  Batch* b = as_batch(h);
  if (b && b->graph) cudaGraphExecDestroy(b->graph);
  delete b;
}

static int lbm_batch_set_stream_body(lbm_batch_handle h, void* stream) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  b->stream = static_cast<cudaStream_t>(stream);
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  return LBM_OK;
}

static int lbm_batch_init_run_body(lbm_batch_handle h, int run, const void* rho, const void* u, int dtype, int on_device) {
  Batch* b = as_batch(h);
  if (int rc = check_run(b, run)) return rc;
  if (b->step != 0) return set_error(LBM_EINVAL, "runs are initialised before the batch takes its first step");
  int rc = lbm_init_fields(reinterpret_cast<lbm_handle>(&b->sims[run]), rho, u, nullptr, dtype, on_device);
  if (!rc) rc = cuda_check(cudaMemsetAsync(b->status() + run, 0, sizeof(int), b->stream), "clear run status");
  return rc;
}

static int lbm_batch_init_runs_body(lbm_batch_handle h, const void* const* rho, const void* const* u, int dtype,
                                    int on_device) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  if (!rho || !u) return set_error(LBM_EINVAL, "NULL field pointer array");
  if (dtype != LBM_DTYPE_F64 && dtype != LBM_DTYPE_F32) return set_error(LBM_EINVAL, "unknown field dtype %d", dtype);
  if (b->step != 0) return set_error(LBM_EINVAL, "runs are initialised before the batch takes its first step");
  for (int r = 0; r < b->n_runs; ++r)
    if (!rho[r] || !u[r]) return set_error(LBM_EINVAL, "NULL field pointer of run %d", r);
  // device-visible views of every run's fields; any pageable array sends all
  // runs through the per-run path (staged copies)
  std::vector<BInitPtrs> table((size_t)b->n_runs);
  bool direct = b->n_runs <= 65535;
  for (int r = 0; r < b->n_runs && direct; ++r) {
    table[r].rho = on_device ? rho[r] : pinned_device_view(rho[r]);
    table[r].u = on_device ? u[r] : pinned_device_view(u[r]);
    direct = table[r].rho && table[r].u;
  }
  if (!direct) {
    for (int r = 0; r < b->n_runs; ++r)
      if (int rc = lbm_batch_init_run_body(h, r, rho[r], u[r], dtype, on_device)) return rc;
    return LBM_OK;
  }
  BInitPtrs* table_dev = reinterpret_cast<BInitPtrs*>(b->work + b->L.init_table);
  int rc = cuda_check(cudaMemcpyAsync(table_dev, table.data(), table.size() * sizeof(BInitPtrs),
                                      cudaMemcpyHostToDevice, b->stream),
                      "upload field table");
  if (!rc) rc = cuda_check(cudaMemsetAsync(b->status(), 0, (size_t)b->n_runs * sizeof(int), b->stream),
                           "clear run status");
  if (!rc) {
    cudaError_t e = cudaErrorInvalidValue;
    switch (b->storage) {
      case LBM_F64: e = launch_batch_init_t<LBM_F64>(b, table_dev, dtype); break;
      case LBM_F32: e = launch_batch_init_t<LBM_F32>(b, table_dev, dtype); break;
      case LBM_F16: e = launch_batch_init_t<LBM_F16>(b, table_dev, dtype); break;
      case LBM_BF16: e = launch_batch_init_t<LBM_BF16>(b, table_dev, dtype); break;
    }
    rc = cuda_check(e, "batch init kernel");
  }
  // the kernel reads the caller's arrays: they are released only once it is done
  if (!rc) rc = cuda_check(cudaStreamSynchronize(b->stream), "stream synchronize");
  if (!rc)
    for (int r = 0; r < b->n_runs; ++r) b->sims[r].step = 0;
  return rc;
}

static int lbm_batch_step_body(lbm_batch_handle h, int64_t n) {
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

static int lbm_batch_use_graph_body(lbm_batch_handle h, int enable) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  b->use_graph = enable != 0;
  return LBM_OK;
}

static int lbm_batch_set_tiles_body(lbm_batch_handle h, int threads, int rows) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  bool okt = false, okr = false;
  for (int t : kThreadChoices) okt = okt || t == threads;
  for (int r : kRowChoices) okr = okr || r == rows;
  if (!okt || !okr) return set_error(LBM_EINVAL, "threads must be 64, 128 or 256 and rows 1, 2, 4, 8 or 16");
  return upload_tiles(b, threads, rows, b->split, b->depth, b->staged);
}

static int lbm_batch_set_launch_body(lbm_batch_handle h, int split, int depth, int staged) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  if ((split != 0 && split != 1) || (depth != 1 && depth != 2) || staged < 0 || staged > stg::kVariants)
    return set_error(LBM_EINVAL, "split must be 0 or 1, depth 1 or 2, staged 0 .. %d", stg::kVariants);
  return upload_tiles(b, b->threads, b->rows, split != 0, depth, staged);
}

static int lbm_batch_get_launch_body(lbm_batch_handle h, int* threads, int* rows, int* split, int* depth, int* staged) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  if (threads) *threads = b->threads;
  if (rows) *rows = b->rows;
  if (split) *split = b->split ? 1 : 0;
  if (depth) *depth = b->depth;
  if (staged) *staged = b->staged;
  return LBM_OK;
}

static int lbm_batch_autotune_body(lbm_batch_handle h, int steps_per_trial, int* threads, int* rows) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  if (b->step != 0) return set_error(LBM_EINVAL, "autotune runs before the first step");
  if (steps_per_trial < 2) return set_error(LBM_EINVAL, "steps_per_trial must be >= 2");
  const std::string key = cache_key(b);
  int bt = 128, br = 1, bs = 0, bd = 1, bg = 1;
  if (!cache_lookup(key, &bt, &br, &bs, &bd, &bg)) {
    // time every launch shape on the rest state (zero offsets), a fixed point of the step
    int rc = cuda_check(cudaMemsetAsync(b->pop, 0, (size_t)b->L.elems * storage_elem_bytes(b->storage), b->stream),
                        "rest state");
    if (rc) return rc;

    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    float best = 1e30f;
    for (int mode = 0; mode < 4 * (1 + stg::kVariants) && !rc; ++mode)
      for (int t : kThreadChoices)
        for (int r : kRowChoices) {
          const int sp = mode & 1, dp = 1 + ((mode >> 1) & 1), sg = mode >> 2;
          if (sg) {
            // with every run staged the tile shape does not matter: one trial
            bool all = true;
            for (int q = 0; q < b->n_runs; ++q) all = all && stage_run(b->storage, sg - 1, b->nx[q]);
            bool any = false;
            for (int q = 0; q < b->n_runs; ++q) any = any || stage_run(b->storage, sg - 1, b->nx[q]);
            if (!any) continue;
            if (all && ((mode & 3) != 0 || t != kThreadChoices[0] || r != kRowChoices[0])) continue;
          }
          rc = upload_tiles(b, t, r, sp != 0, dp, sg);
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
            bs = sp;
            bd = dp;
            bg = sg;
          }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    // the trials took an even number of steps from the rest state: still at rest, parity even
    rc = cuda_check(cudaMemsetAsync(b->pop, 0, (size_t)b->L.elems * storage_elem_bytes(b->storage), b->stream),
                    "rest state");
    if (rc) return rc;
    cache_store(key, bt, br, bs, bd, bg);
  }
  if (threads) *threads = bt;
  if (rows) *rows = br;
  return upload_tiles(b, bt, br, bs != 0, bd, bg);
}

static int lbm_batch_status_body(lbm_batch_handle h, int* flags) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  if (!flags) return set_error(LBM_EINVAL, "NULL output pointer");
  std::vector<int> st(b->n_runs);
  int rc = cuda_check(cudaMemcpyAsync(st.data(), b->status(), st.size() * sizeof(int), cudaMemcpyDeviceToHost,
                                      b->stream),
                      "status readback");
  if (!rc) rc = cuda_check(cudaStreamSynchronize(b->stream), "stream synchronize");
  if (rc) return rc;
  for (int r = 0; r < b->n_runs; ++r) flags[r] = (st[r] & 2) ? LBM_ETIMEOUT : (st[r] ? LBM_EDIVERGED : LBM_OK);
  return LBM_OK;
}

static int lbm_batch_reduce_body(lbm_batch_handle h, double* out) {
  Batch* b = as_batch(h);
  if (int rc = check_batch(b)) return rc;
  if (!out) return set_error(LBM_EINVAL, "NULL output pointer");
  // one launch for every run: block r sums run r
  bool launched = true;
  const int odd = (int)(b->step & 1);
  switch (b->storage) {
    case LBM_F64: batch_reduce_kernel<LBM_F64><<<b->n_runs, kAuxThreads, 0, b->stream>>>(
                      static_cast<const double*>(b->pop), b->runs_dev(), odd, b->results()); break;
    case LBM_F32: batch_reduce_kernel<LBM_F32><<<b->n_runs, kAuxThreads, 0, b->stream>>>(
                      static_cast<const float*>(b->pop), b->runs_dev(), odd, b->results()); break;
    case LBM_F16: batch_reduce_kernel<LBM_F16><<<b->n_runs, kAuxThreads, 0, b->stream>>>(
                      static_cast<const __half*>(b->pop), b->runs_dev(), odd, b->results()); break;
    case LBM_BF16: batch_reduce_kernel<LBM_BF16><<<b->n_runs, kAuxThreads, 0, b->stream>>>(
                      static_cast<const __nv_bfloat16*>(b->pop), b->runs_dev(), odd, b->results()); break;
    default: launched = false;
  }
  int rc = launched ? cuda_check(cudaGetLastError(), "run totals") : set_error(LBM_EINVAL, "unknown storage");
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

static int lbm_batch_moments_body(lbm_batch_handle h, int run, void* rho, void* u, int dtype, int on_device) {
  Batch* b = as_batch(h);
  if (int rc = check_run(b, run)) return rc;
  return lbm_moments(reinterpret_cast<lbm_handle>(&b->sims[run]), rho, u, nullptr, dtype, on_device);
}

static int lbm_batch_get_populations_body(lbm_batch_handle h, int run, double* f, int on_device) {
  Batch* b = as_batch(h);
  if (int rc = check_run(b, run)) return rc;
  return lbm_get_populations(reinterpret_cast<lbm_handle>(&b->sims[run]), f, on_device);
}

int64_t lbm_batch_step_count(lbm_batch_handle h) {
  Batch* b = as_batch(h);
  return b ? b->step : -1;
}


int lbm_batch_query_bytes(int lattice, int n_runs, const int64_t* dims, int storage, size_t* pop_bytes,
                          size_t* work_bytes) {
  return host_guard("lbm_batch_query_bytes", [&] { return lbm_batch_query_bytes_body(lattice, n_runs, dims, storage, pop_bytes, work_bytes); });
}

int lbm_batch_create(int lattice, int n_runs, const int64_t* dims, const double* tau_per_order, int n_tau,
                     int storage, void* pop, size_t pop_bytes, void* work, size_t work_bytes,
                     lbm_batch_handle* out) {
  return host_guard("lbm_batch_create", [&] { return lbm_batch_create_body(lattice, n_runs, dims, tau_per_order, n_tau, storage, pop, pop_bytes, work, work_bytes, out); });
}

int lbm_batch_set_stream(lbm_batch_handle h, void* stream) {
  return host_guard("lbm_batch_set_stream", [&] { return lbm_batch_set_stream_body(h, stream); });
}

int lbm_batch_init_run(lbm_batch_handle h, int run, const void* rho, const void* u, int dtype, int on_device) {
  return host_guard("lbm_batch_init_run", [&] { return lbm_batch_init_run_body(h, run, rho, u, dtype, on_device); });
}

int lbm_batch_init_runs(lbm_batch_handle h, const void* const* rho, const void* const* u, int dtype, int on_device) {
  return host_guard("lbm_batch_init_runs", [&] { return lbm_batch_init_runs_body(h, rho, u, dtype, on_device); });
}

int lbm_batch_step(lbm_batch_handle h, int64_t n) {
  return host_guard("lbm_batch_step", [&] { return lbm_batch_step_body(h, n); });
}

int lbm_batch_use_graph(lbm_batch_handle h, int enable) {
  return host_guard("lbm_batch_use_graph", [&] { return lbm_batch_use_graph_body(h, enable); });
}

int lbm_batch_set_tiles(lbm_batch_handle h, int threads, int rows) {
  return host_guard("lbm_batch_set_tiles", [&] { return lbm_batch_set_tiles_body(h, threads, rows); });
}

int lbm_batch_set_launch(lbm_batch_handle h, int split, int depth, int staged) {
  return host_guard("lbm_batch_set_launch", [&] { return lbm_batch_set_launch_body(h, split, depth, staged); });
}

int lbm_batch_get_launch(lbm_batch_handle h, int* threads, int* rows, int* split, int* depth, int* staged) {
  return host_guard("lbm_batch_get_launch", [&] { return lbm_batch_get_launch_body(h, threads, rows, split, depth, staged); });
}

int lbm_batch_autotune(lbm_batch_handle h, int steps_per_trial, int* threads, int* rows) {
  return host_guard("lbm_batch_autotune", [&] { return lbm_batch_autotune_body(h, steps_per_trial, threads, rows); });
}

int lbm_batch_status(lbm_batch_handle h, int* flags) {
  return host_guard("lbm_batch_status", [&] { return lbm_batch_status_body(h, flags); });
}

int lbm_batch_reduce(lbm_batch_handle h, double* out) {
  return host_guard("lbm_batch_reduce", [&] { return lbm_batch_reduce_body(h, out); });
}

int lbm_batch_moments(lbm_batch_handle h, int run, void* rho, void* u, int dtype, int on_device) {
  return host_guard("lbm_batch_moments", [&] { return lbm_batch_moments_body(h, run, rho, u, dtype, on_device); });
}

int lbm_batch_get_populations(lbm_batch_handle h, int run, double* f, int on_device) {
  return host_guard("lbm_batch_get_populations", [&] { return lbm_batch_get_populations_body(h, run, f, on_device); });
}

}  // extern "C"
