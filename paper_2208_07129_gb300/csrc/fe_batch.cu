// Batched uneven workload: many operators (different meshes, degrees and
// block widths) applied by ONE persistent kernel, launched from a CUDA graph.
//
// Work items are (problem, colour, range of cells of that colour, vector
// block).  The queue is ordered by colour phase first (all problems' colour-0
// items, then colour 1, ...), so an item of colour k > 0 of problem i only has
// to wait until every colour k-1 item of problem i is done; those were taken
// from the queue earlier by running CTAs, so the wait always ends (and it is
// bounded besides: a CTA that gives up records FE_ETIMEOUT).  Within a colour
// the cells share no node, so assembly stays conflict-free and the result is
// bitwise the one of the per-problem launches of the even-odd line kernel
// (the same cell body; Sec. 3.1.2: all cells and batches of vectors evaluated
// concurrently, here across problems too).
//
// Each problem gets its own tile (vectors per item x lines per CTA, 128
// threads) from a small autotuner that times the candidate tiles on a proxy
// mesh of the same degree and block width, and a cell-batch size (cells per
// item) that keeps the queue several items deep per SM.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <vector>

#include <type_traits>

#include "fe_internal.h"
#include "fe_cell_kernel.cuh"
#include "fe_dispatch.cuh"
#include "fe_evenodd.cuh"
#include "fe_ff_body.cuh"
#include "../../include/fe_batch.h"

namespace fe {

constexpr int kBatchThreads = 128;
constexpr int kMaxColors = 27;
constexpr int kTabImage = 256;   // elements of an EOTables<T, NP, NQ> image (195 at p = 8, n_q = 10)
constexpr int kKinds = 6;        // degrees 3..8 with n_q = p + 2

template <typename T>
struct BatchProblemDev {
  MeshDev m;
  Geom<T> geo;
  int n_vec, vb, nty, kind, n_vb;
  const int* cells;                                    // colour-sorted cell ids
  T tab[kTabImage];                                    // EOTables<T, NP, NQ> image
};

struct WorkItem {
  int problem, color, cell_begin, cell_count, vb;
};

// Element type of X and Y for a compute type (double-float computes on FP64 data).
template <typename T>
struct DataOf { using type = T; };
template <>
struct DataOf<ff> { using type = double; };

// kinds: p = 3..8 with n_q = p + 2 on affine cells
constexpr int kind_of(int p) { return p - 3; }

template <typename T, int NP, int NQ>
__device__ __forceinline__ void run_item(const BatchProblemDev<T>& P, const WorkItem& w,
                                         const typename DataOf<T>::type* X, typename DataOf<T>::type* Y, T* smem,
                                         const EOTables<T, NP, NQ>& tab) {
  const int tid = threadIdx.x, vb = P.vb;
  const int v = tid % vb, ty = tid / vb, nty = kBatchThreads / vb;
  for (int c = 0; c < w.cell_count; ++c) {
    const int e = P.cells[w.cell_begin + c];
    if constexpr (std::is_same<T, ff>::value)
      cell_body_ff<NP, NQ, false, false>(tab, P.m, P.geo, e, w.vb, vb, v, ty, nty, P.n_vec, X, Y, smem,
                                         Scale<double>{});
    else
      cell_body_eo<T, NP, NQ, false>(tab, P.m, P.geo, e, w.vb, vb, v, ty, nty, P.n_vec, X, Y, smem);
    __syncthreads();
  }
}

__device__ __forceinline__ unsigned long long batch_clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// One persistent kernel per degree (the problems of that degree, their own
// queue): each instantiation gets the registers its cell body needs instead
// of those of the largest degree in the batch, and the degree's 1D tables
// (the same for all its problems) travel as a kernel parameter, so the
// contractions read their coefficients from the constant bank as in the
// per-colour kernels.
template <typename T, int NP, int NQ>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel(const EOTables<T, NP, NQ> tab,
                                                             const BatchProblemDev<T>* __restrict__ probs,
                                                             const void* const* __restrict__ ptrs,
                                                             const WorkItem* __restrict__ items, int n_items,
                                                             int* next, int* done, const int* __restrict__ need,
                                                             int* status, const long long* __restrict__ wait_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_item;
  T* smem = reinterpret_cast<T*>(smem_raw);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const WorkItem w = items[it];
    const BatchProblemDev<T>& P = probs[w.problem];
    if (threadIdx.x == 0 && w.color > 0) {
      const int idx = w.problem * kMaxColors + w.color - 1;
      const long long limit = *wait_ns;
      const long long t0 = (long long)batch_clock_ns();
      while (atomicAdd(&done[idx], 0) < need[idx]) {
        __nanosleep(128);
        if ((long long)batch_clock_ns() - t0 > limit) {
          atomicMax(status, (int)FE_ETIMEOUT);
          break;
        }
      }
      __threadfence();
    }
    __syncthreads();
    using D = typename DataOf<T>::type;
    const D* X = static_cast<const D*>(ptrs[2 * w.problem]);
    D* Y = static_cast<D*>(const_cast<void*>(ptrs[2 * w.problem + 1]));
    run_item<T, NP, NQ>(P, w, X, Y, smem, tab);
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&done[w.problem * kMaxColors + w.color], 1);
    }
    __syncthreads();
  }
}


// FP64: one persistent kernel for every degree, the tables of each item's
// problem staged in shared memory.  Measured faster than the per-degree
// kernels for FP64 (950 against 1030 ms on the 24-problem batch): the FP64
// pipe bounds both, and one kernel keeps every degree's work in flight
// together.  Its register allocation is the largest degree's, which costs the
// double-float and FP32 cell bodies much more than it costs FP64.
template <typename T>
__global__ void __launch_bounds__(kBatchThreads) batch_kernel_all(const BatchProblemDev<T>* __restrict__ probs,
                                                                 const void* const* __restrict__ ptrs,
                                                                 const WorkItem* __restrict__ items, int n_items,
                                                                 int* next, int* done, const int* __restrict__ need,
                                                                 int* status, const long long* __restrict__ wait_ns) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) T stab[kTabImage];
  __shared__ int s_item;
  T* smem = reinterpret_cast<T*>(smem_raw);
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items) break;
    const WorkItem w = items[it];
    const BatchProblemDev<T>& P = probs[w.problem];
    if (threadIdx.x == 0 && w.color > 0) {
      const int idx = w.problem * kMaxColors + w.color - 1;
      const long long limit = *wait_ns;
      const long long t0 = (long long)batch_clock_ns();
      while (atomicAdd(&done[idx], 0) < need[idx]) {
        __nanosleep(128);
        if ((long long)batch_clock_ns() - t0 > limit) {
          atomicMax(status, (int)FE_ETIMEOUT);
          break;
        }
      }
      __threadfence();
    }
    for (int k = threadIdx.x; k < kTabImage; k += blockDim.x) stab[k] = P.tab[k];
    __syncthreads();
    using D = typename DataOf<T>::type;
    const D* X = static_cast<const D*>(ptrs[2 * w.problem]);
    D* Y = static_cast<D*>(const_cast<void*>(ptrs[2 * w.problem + 1]));
#define FE_ITEM(K, NP, NQ) \
  case K: run_item<T, NP, NQ>(P, w, X, Y, smem, *reinterpret_cast<const EOTables<T, NP, NQ>*>(stab)); break;
    switch (P.kind) {
      FE_ITEM(0, 4, 5) FE_ITEM(1, 5, 6) FE_ITEM(2, 6, 7) FE_ITEM(3, 7, 8) FE_ITEM(4, 8, 9) FE_ITEM(5, 9, 10)
      default: break;
    }
#undef FE_ITEM
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&done[w.problem * kMaxColors + w.color], 1);
    }
    __syncthreads();
  }
}

}  // namespace fe

using namespace fe;

struct fe_batch {
  int n = 0;
  fe_mode mode = FE_FP64;
  std::vector<fe_ctx*> ctxs;
  std::vector<int> n_vec, vb, cells_per_item;
  void* d_probs = nullptr;
  WorkItem* d_items = nullptr;
  int n_items = 0, n_phases = 0;
  int item_begin[kKinds + 1] = {0};   // items of degree kind k: [item_begin[k], item_begin[k + 1])
  int *d_next = nullptr, *d_done = nullptr, *d_need = nullptr, *d_status = nullptr;
  std::vector<int> need;               // host copy of the completion counts items wait for
  long long* d_wait_ns = nullptr;      // limit of one bounded wait (device, read by the kernels)
  const void** h_ptrs = nullptr;   // pinned host staging of the X / Y table
  void** d_ptrs = nullptr;
  size_t smem = 0;
  int grid = 0;
  int grid_kind[kKinds] = {0};         // persistent grid of each degree's kernel (per-degree kernels)
  cudaStream_t cap = nullptr;
  cudaStream_t side[kKinds] = {};       // one capture branch per degree
  cudaEvent_t fork = nullptr, join[kKinds] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  float tune_ms = 0.f;
};

namespace {

fe_status from_cuda(cudaError_t e) {
  return fe::cuda_status(e);
}

template <typename T>
size_t tile_smem(int nq, int vb) { return (size_t)3 * nq * nq * nq * vb * sizeof(T); }

// The even-odd tables of one problem, copied into its table image.
template <typename T, int NP, int NQ>
void eo_image(const fe_ctx* c, T* img) {
  static_assert(sizeof(EOTables<T, NP, NQ>) <= kTabImage * sizeof(T), "table image too small");
  const EOTables<T, NP, NQ> t = make_eotables<T, NP, NQ>(c);
  std::memcpy(img, &t, sizeof(t));
}

// Candidate vectors-per-CTA of the autotuner for one problem.
std::vector<int> candidates(int nq, int n_vec, size_t elem) {
  std::vector<int> out;
  for (int vb : {2, 4, 8, 16, 32}) {
    if ((size_t)3 * nq * nq * nq * vb * elem > 110 * 1024) continue;   // keep two CTAs per SM
    if (vb > 1 && vb / 2 >= n_vec) continue;
    out.push_back(vb);
  }
  if (out.empty()) out.push_back(2);
  return out;
}

// Time one apply of an 8^3 periodic proxy (64 cells per colour: enough CTAs
// to fill the GPU at every candidate, unlike a tiny mesh, which rewards the
// narrowest tile for its parallelism alone) with the problem's degree and
// block width (capped at 64 vectors) for every candidate tile; return the
// fastest vectors-per-CTA.
int autotune(const fe_ctx* c, int n_vec_full, fe_mode mode, float* spent_ms) {
  const size_t elem = mode == FE_FP32 ? 4 : 8;
  std::vector<int> cand = candidates(c->nq, n_vec_full, elem);
  if (cand.size() == 1) return cand[0];
  const int n_vec = std::min(n_vec_full, 64);
  fe_mesh_desc md{};
  md.nx = md.ny = md.nz = 8;
  md.hi[0] = md.hi[1] = md.hi[2] = 1.0;
  md.bc = FE_BC_PERIODIC;
  fe_quad_desc qd{c->nq, c->quad_kind};
  fe_ctx* px = nullptr;
  if (fe_setup(&md, c->p, &qd, c->mu, &px) != FE_OK) return cand[0];
  fe_set_mode(px, mode);
  const size_t bytes = px->n_dofs * (size_t)n_vec * elem;
  void *X = nullptr, *Y = nullptr;
  int best = cand[0];
  if (cudaMalloc(&X, bytes) == cudaSuccess && cudaMalloc(&Y, bytes) == cudaSuccess) {
    cudaMemset(X, 0, bytes);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best_ms = 1e30f;
    for (int vb : cand) {
      fe_set_tile(px, mode, vb, kBatchThreads / vb, mode == FE_FP32 ? 3 : 0);   // the even-odd line kernel
      fe_apply(px, X, Y, n_vec, nullptr);
      cudaEventRecord(a);
      for (int r = 0; r < 3; ++r) fe_apply(px, X, Y, n_vec, nullptr);
      cudaEventRecord(b);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      *spent_ms += ms;
      if (ms < best_ms) { best_ms = ms; best = vb; }
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
  cudaFree(X);
  cudaFree(Y);
  fe_destroy(px);
  cudaGetLastError();
  return best;
}

// The persistent kernel of one degree: before the capture, its shared-memory
// attribute and its grid = occupancy x SMs (at most one CTA per work item);
// then its launch, recorded into the graph.
template <typename T, int NP, int NQ>
cudaError_t prepare_kind(fe_batch* b, int kind, int n_k, size_t smem) {
  auto kern = batch_kernel<T, NP, NQ>;
  cudaError_t e = ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  int per_sm = 0, sms = 0, dev = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  b->grid_kind[kind] = std::max(1, std::min(n_k, std::max(1, per_sm) * sms));
  b->grid = std::max(b->grid, b->grid_kind[kind]);
  return cudaSuccess;
}

template <typename T, int NP, int NQ>
cudaError_t launch_kind(fe_batch* b, int kind, int n_k, size_t smem) {
  auto kern = batch_kernel<T, NP, NQ>;
  const fe_ctx* c0 = nullptr;   // the degree's tables: those of its first problem (all equal)
  for (int i = 0; i < b->n && !c0; ++i)
    if (kind_of(b->ctxs[i]->p) == kind) c0 = b->ctxs[i];
  if (!c0) return cudaErrorInvalidValue;
  const EOTables<T, NP, NQ> tab = make_eotables<T, NP, NQ>(c0);
  kern<<<b->grid_kind[kind], kBatchThreads, smem, b->side[kind]>>>(
      tab, static_cast<const BatchProblemDev<T>*>(b->d_probs), const_cast<const void* const*>(b->d_ptrs),
      b->d_items + b->item_begin[kind], n_k, b->d_next + kind, b->d_done, b->d_need, b->d_status, b->d_wait_ns);
  return cudaGetLastError();
}

// Both steps for kind k (p = k + 3, n_q = p + 2).
template <typename T>
cudaError_t for_kind(fe_batch* b, int kind, int n_k, size_t smem, bool launch) {
  switch (kind) {
    case 0: return launch ? launch_kind<T, 4, 5>(b, kind, n_k, smem) : prepare_kind<T, 4, 5>(b, kind, n_k, smem);
    case 1: return launch ? launch_kind<T, 5, 6>(b, kind, n_k, smem) : prepare_kind<T, 5, 6>(b, kind, n_k, smem);
    case 2: return launch ? launch_kind<T, 6, 7>(b, kind, n_k, smem) : prepare_kind<T, 6, 7>(b, kind, n_k, smem);
    case 3: return launch ? launch_kind<T, 7, 8>(b, kind, n_k, smem) : prepare_kind<T, 7, 8>(b, kind, n_k, smem);
    case 4: return launch ? launch_kind<T, 8, 9>(b, kind, n_k, smem) : prepare_kind<T, 8, 9>(b, kind, n_k, smem);
    case 5: return launch ? launch_kind<T, 9, 10>(b, kind, n_k, smem) : prepare_kind<T, 9, 10>(b, kind, n_k, smem);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
fe_status build_batch(fe_batch* b, int autotune_on) {
  const int n = b->n;
  std::vector<BatchProblemDev<T>> hp(n);
  std::vector<int> need((size_t)n * kMaxColors, 0);
  std::map<std::pair<int, int>, int> tuned;   // (p, n_vec bucket) -> vb
  size_t smem = 0;
  long long total_units = 0;
  for (int i = 0; i < n; ++i) total_units += (long long)b->ctxs[i]->n_cells * ((b->n_vec[i] + 7) / 8);
  for (int i = 0; i < n; ++i) {
    fe_ctx* c = b->ctxs[i];
    BatchProblemDev<T>& P = hp[i];
    P.m = c->mdev;
    if constexpr (std::is_same<T, ff>::value) P.geo = Geom<ff>{c->d_cellGff, c->d_ptGff, c->d_ptCff};
    else if (b->mode == FE_FP64) P.geo = Geom<T>{(const T*)c->d_cellG64, (const T*)c->d_ptG64, (const T*)c->d_ptC64};
    else P.geo = Geom<T>{(const T*)c->d_cellG32, (const T*)c->d_ptG32, (const T*)c->d_ptC32};
    P.n_vec = b->n_vec[i];
    P.kind = kind_of(c->p);
    P.cells = c->d_cells;
    const int bucket = (int)std::ceil(std::log2((double)std::max(1, P.n_vec)));
    int vb;
    auto key = std::make_pair(c->p, bucket);
    if (!autotune_on) {
      vb = candidates(c->nq, P.n_vec, sizeof(T)).back();
      vb = std::min(vb, 8);
    } else if (tuned.count(key)) {
      vb = tuned[key];
    } else {
      vb = autotune(c, P.n_vec, b->mode, &b->tune_ms);
      tuned[key] = vb;
    }
    P.vb = vb;
    P.nty = kBatchThreads / vb;
    P.n_vb = (P.n_vec + vb - 1) / vb;
    b->vb[i] = vb;
    std::memset(P.tab, 0, sizeof(P.tab));
    switch (P.kind) {
      case 0: eo_image<T, 4, 5>(c, P.tab); break;
      case 1: eo_image<T, 5, 6>(c, P.tab); break;
      case 2: eo_image<T, 6, 7>(c, P.tab); break;
      case 3: eo_image<T, 7, 8>(c, P.tab); break;
      case 4: eo_image<T, 8, 9>(c, P.tab); break;
      case 5: eo_image<T, 9, 10>(c, P.tab); break;
      default: break;
    }
    smem = std::max(smem, tile_smem<T>(c->nq, vb));
  }
  // work items, phase-major: one queue over all problems (FP64, merged
  // kernel) or one queue per degree (per-degree kernels)
  constexpr bool merged = std::is_same<T, double>::value;
  std::vector<WorkItem> items;
  int phases = 0;
  for (int kind = 0; kind < (merged ? 1 : kKinds); ++kind) {
  b->item_begin[kind] = (int)items.size();
  for (int k = 0; k < kMaxColors; ++k) {
    bool any = false;
    for (int i = 0; i < n; ++i) {
      fe_ctx* c = b->ctxs[i];
      if ((!merged && hp[i].kind != kind) || k >= c->colors.n_colors) continue;
      any = true;
      const int c0 = c->colors.offset[k], c1 = c->colors.offset[k + 1];
      const BatchProblemDev<T>& P = hp[i];
      // cells per item: keep >= ~8 items per SM over the whole batch
      const long long per_color = (long long)(c1 - c0) * P.n_vb;
      int cb = 1;
      while (cb < 8 && per_color / (2 * cb) >= 64 && total_units / (2 * cb) > 152 * 32) cb *= 2;
      b->cells_per_item[i] = cb;
      for (int s = c0; s < c1; s += cb)
        for (int v = 0; v < P.n_vb; ++v) {
          items.push_back(WorkItem{i, k, s, std::min(cb, c1 - s), v});
          need[(size_t)i * kMaxColors + k]++;
        }
    }
    if (any) phases = std::max(phases, k + 1);
  }
  }
  for (int kind = merged ? 1 : kKinds; kind <= kKinds; ++kind) b->item_begin[kind] = (int)items.size();
  b->n_items = (int)items.size();
  b->n_phases = phases;
  b->smem = smem;
  const char* where = "fe_batch_create: device tables";
  cudaError_t e = cudaMalloc(&b->d_probs, n * sizeof(BatchProblemDev<T>));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_probs, hp.data(), n * sizeof(BatchProblemDev<T>), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_items, std::max<size_t>(1, items.size()) * sizeof(WorkItem));
  if (e == cudaSuccess && !items.empty())
    e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(WorkItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_need, need.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMemcpy(b->d_need, need.data(), need.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&b->d_done, need.size() * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_next, kKinds * sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(b->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMalloc(&b->d_wait_ns, sizeof(long long));
  if (e == cudaSuccess) {
    const long long ten_s = 10000000000LL;
    e = cudaMemcpy(b->d_wait_ns, &ten_s, sizeof(long long), cudaMemcpyHostToDevice);
  }
  b->need = need;
  if (e == cudaSuccess) e = cudaMalloc(&b->d_ptrs, 2 * n * sizeof(void*));
  if (e == cudaSuccess) e = cudaMallocHost(&b->h_ptrs, 2 * n * sizeof(void*));
  if (e != cudaSuccess) return fe::cuda_status(e, where);
  // graph: reset the queues and the colour counters, then one persistent
  // kernel per degree present, as parallel branches (the degrees share the
  // GPU, and one degree's tail overlaps the others' work).  Every wait of a
  // CTA is on items its own kernel dequeued earlier, whose CTAs are running,
  // so concurrent branches cannot block each other.
  // kernel attributes and grids first: the capture below only records work
  where = "fe_batch_create: kernel attributes and grids";
  if constexpr (merged) {
    auto kern = batch_kernel_all<T>;
    e = ensure_dyn_smem(reinterpret_cast<const void*>(kern), smem);
    int per_sm = 0, sms = 0, dev = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBatchThreads, smem);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    b->grid = std::max(1, std::min(b->n_items, std::max(1, per_sm) * sms));
  } else {
    for (int kind = 0; kind < kKinds && e == cudaSuccess; ++kind) {
      const int n_k = b->item_begin[kind + 1] - b->item_begin[kind];
      if (n_k > 0) e = for_kind<T>(b, kind, n_k, smem, false);
    }
  }
  if (e != cudaSuccess) return fe::cuda_status(e, where);
  where = "fe_batch_create: streams and events";
  e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
  for (int k = 0; k < kKinds && e == cudaSuccess; ++k) e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int k = 0; k < kKinds && e == cudaSuccess; ++k) e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    where = "fe_batch_create: captured launches";
    cudaMemsetAsync(b->d_next, 0, kKinds * sizeof(int), b->cap);
    cudaMemsetAsync(b->d_done, 0, need.size() * sizeof(int), b->cap);
    cudaEventRecord(b->fork, b->cap);
    if constexpr (merged) {
      batch_kernel_all<T><<<b->grid, kBatchThreads, smem, b->cap>>>(
          static_cast<const BatchProblemDev<T>*>(b->d_probs), const_cast<const void* const*>(b->d_ptrs), b->d_items,
          b->n_items, b->d_next, b->d_done, b->d_need, b->d_status, b->d_wait_ns);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      e = cudaGetLastError();
      if (e != cudaSuccess) where = "fe_batch_create: captured resets of the queues";
    }
    for (int kind = 0; kind < kKinds && e == cudaSuccess && !merged; ++kind) {
      const int n_k = b->item_begin[kind + 1] - b->item_begin[kind];
      if (n_k == 0) continue;
      e = cudaStreamWaitEvent(b->side[kind], b->fork, 0);
      if (e != cudaSuccess) { where = "fe_batch_create: fork of a degree's branch"; break; }
      e = for_kind<T>(b, kind, n_k, smem, true);
      if (e != cudaSuccess) { where = "fe_batch_create: captured launch of a degree's kernel"; break; }
      e = cudaEventRecord(b->join[kind], b->side[kind]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap, b->join[kind], 0);
      if (e != cudaSuccess) where = "fe_batch_create: join of a degree's branch";
    }
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    b->graph = g;
    if (e == cudaSuccess && e2 != cudaSuccess) where = "fe_batch_create: end of capture";
    if (e == cudaSuccess) e = e2;
  }
  if (e == cudaSuccess) {
    where = "fe_batch_create: graph instantiation";
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  }
  return fe::cuda_status(e, where);
}

}  // namespace

extern "C" fe_status fe_batch_create(fe_ctx* const* ctxs, int n, const int* n_vec, fe_mode mode, int autotune_on,
                                     fe_batch** out) {
  if (!out) return FE_EINVAL;
  *out = nullptr;
  if (!ctxs || !n_vec || n <= 0) return FE_EINVAL;
  if (mode != FE_FP64 && mode != FE_FP32 && mode != FE_DF64) return FE_EUNSUPPORTED;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || n_vec[i] <= 0) return FE_EINVAL;
    if (ctxs[i]->general || ctxs[i]->refined || ctxs[i]->p < 3 || ctxs[i]->p > 8 || ctxs[i]->nq != ctxs[i]->p + 2)
      return FE_EUNSUPPORTED;
    for (int j = 0; j < i; ++j)   // one quadrature rule per degree: the degree's kernel carries one set of tables
      if (ctxs[j]->p == ctxs[i]->p && ctxs[j]->quad_kind != ctxs[i]->quad_kind) return FE_EUNSUPPORTED;
  }
  fe_batch* b = new fe_batch();
  b->n = n;
  b->mode = mode;
  b->ctxs.assign(ctxs, ctxs + n);
  b->n_vec.assign(n_vec, n_vec + n);
  b->vb.assign(n, 0);
  b->cells_per_item.assign(n, 1);
  fe_status st = mode == FE_FP64 ? build_batch<double>(b, autotune_on)
                 : mode == FE_DF64 ? build_batch<ff>(b, autotune_on)
                                   : build_batch<float>(b, autotune_on);
  if (st != FE_OK) {
    fe_batch_destroy(b);
    return st;
  }
  *out = b;
  return FE_OK;
}

extern "C" fe_status fe_batch_apply(fe_batch* b, const void* const* X, void* const* Y, void* stream) {
  if (!b || !X || !Y) return FE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  for (int i = 0; i < b->n; ++i) {
    if (!X[i] || !Y[i] || X[i] == Y[i]) return FE_EINVAL;
    b->h_ptrs[2 * i] = X[i];
    b->h_ptrs[2 * i + 1] = Y[i];
  }
  // the table is read by the kernel of this launch; wait for the previous use of the staging buffer
  cudaError_t e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_ptrs, b->h_ptrs, 2 * b->n * sizeof(void*), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, s);
  return from_cuda(e);
}

extern "C" fe_status fe_batch_stats(const fe_batch* b, fe_batch_info* info, int* vectors_per_cta, int* cells_per_item) {
  if (!b || !info) return FE_EINVAL;
  info->problems = b->n;
  info->work_items = b->n_items;
  info->phases = b->n_phases;
  info->grid = b->grid;
  info->smem_bytes = (long long)b->smem;
  info->autotune_ms = b->tune_ms;
  for (int i = 0; i < b->n; ++i) {
    if (vectors_per_cta) vectors_per_cta[i] = b->vb[i];
    if (cells_per_item) cells_per_item[i] = b->cells_per_item[i];
  }
  int h = 0;
  if (cudaDeviceSynchronize() != cudaSuccess || cudaMemcpy(&h, b->d_status, sizeof(int), cudaMemcpyDeviceToHost) !=
                                                    cudaSuccess)
    return FE_ECUDA;
  info->device_status = h;
  cudaMemset(b->d_status, 0, sizeof(int));
  return FE_OK;
}

extern "C" fe_status fe_batch_set_wait_limit(fe_batch* b, double seconds) {
  if (!b || !(seconds > 0.0) || seconds > 3600.0) return FE_EINVAL;
  const long long ns = (long long)(seconds * 1e9);
  return from_cuda(cudaMemcpy(b->d_wait_ns, &ns, sizeof(long long), cudaMemcpyHostToDevice));
}

extern "C" fe_status fe_batch_hold_color(fe_batch* b, int problem, int color, int hold) {
  if (!b || problem < 0 || problem >= b->n || color < 0 || color + 1 >= kMaxColors) return FE_EINVAL;
  const size_t idx = (size_t)problem * kMaxColors + color;
  if (b->need[idx] == 0) return FE_EINVAL;   // no work item of that colour, nothing waits for it
  const int v = hold ? 0x7fffffff : b->need[idx];
  return from_cuda(cudaMemcpy(b->d_need + idx, &v, sizeof(int), cudaMemcpyHostToDevice));
}

extern "C" void fe_batch_destroy(fe_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap) cudaStreamDestroy(b->cap);
  for (int k = 0; k < kKinds; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->join[k]) cudaEventDestroy(b->join[k]);
  }
  if (b->fork) cudaEventDestroy(b->fork);
  cudaFree(b->d_probs); cudaFree(b->d_items); cudaFree(b->d_need); cudaFree(b->d_done); cudaFree(b->d_next);
  cudaFree(b->d_status); cudaFree(b->d_ptrs); cudaFree(b->d_wait_ns);
  if (b->h_ptrs) cudaFreeHost(b->h_ptrs);
  delete b;
}
