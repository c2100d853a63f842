// Mixed-degree meshes: p-binned persistent launch, CUDA graph replay and the
// tile-shape autotuner.
//
// The paper's host code first classifies the elements by degree (Section 4.2)
// and then sizes one kernel per class.  Here the classes become bins of a
// single work list: a plan sorts the elements by degree on the host, cuts each
// bin into work items (a group of elements of one degree x one output tile)
// and orders the items by decreasing cost, so that one persistent launch, in
// which every CTA pulls the next item from an atomic counter, balances the
// expensive high-degree elements against the cheap ones.  The counter reset
// and the launch are captured once in a CUDA graph and replayed.  Each degree
// has two candidate tile shapes for the persistent kernel; the autotuner times
// both on the plan's own elements (the first execution) and keeps the faster,
// optionally caching the choice in a text file.  The per-degree modes (a
// launch loop, or one graph branch per degree) run one specialised launch per
// bin and add a third candidate, the degree's uniform-degree kernel, timed the
// same way.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <mutex>
#include <new>
#include <sstream>
#include <string>
#include <vector>

#include "fem_fma.cuh"
#include "fem_internal.h"

namespace fem {

constexpr int kBatchThreads = 256;
constexpr int kVariants = 2;   // candidate shapes of the persistent kernel
// Per-degree launches (loop and concurrent-branch plans) have a third
// candidate: the degree's uniform-degree kernel (no 256-thread limit).
constexpr int kStandalone = 2;
// Plans with a tensor-core precision (per-degree modes only) have a fourth:
// the tensor-core kernel; their FMA candidates run in FP32.
constexpr int kTensor = 3;
constexpr int kMaxVariants = 4;

// Candidate shapes (ELEM, P, BM, TM, TN, EPB, QC), all with at most 256 threads.
template <int P, int V> struct BShape;
template <> struct BShape<1, 0> { using type = FmaCfg<FEM_PRISM6, 1, 6, 1, 6, 42, 4>; };
template <> struct BShape<1, 1> { using type = FmaCfg<FEM_PRISM6, 1, 6, 2, 3, 42, 8>; };
template <> struct BShape<2, 0> { using type = FmaCfg<FEM_PRISM6, 2, 18, 3, 6, 14, 3>; };
template <> struct BShape<2, 1> { using type = FmaCfg<FEM_PRISM6, 2, 18, 6, 6, 28, 3>; };
template <> struct BShape<3, 0> { using type = FmaCfg<FEM_PRISM6, 3, 40, 4, 4, 2, 8>; };
template <> struct BShape<3, 1> { using type = FmaCfg<FEM_PRISM6, 3, 40, 5, 5, 4, 4>; };
template <> struct BShape<4, 0> { using type = FmaCfg<FEM_PRISM6, 4, 75, 5, 5, 1, 5>; };
template <> struct BShape<4, 1> { using type = FmaCfg<FEM_PRISM6, 4, 40, 4, 4, 2, 8>; };
template <> struct BShape<5, 0> { using type = FmaCfg<FEM_PRISM6, 5, 64, 4, 4, 1, 8>; };
template <> struct BShape<5, 1> { using type = FmaCfg<FEM_PRISM6, 5, 63, 7, 7, 3, 4>; };
template <> struct BShape<6, 0> { using type = FmaCfg<FEM_PRISM6, 6, 98, 7, 7, 1, 7>; };
template <> struct BShape<6, 1> { using type = FmaCfg<FEM_PRISM6, 6, 52, 4, 4, 1, 8>; };
template <> struct BShape<7, 0> { using type = FmaCfg<FEM_PRISM6, 7, 96, 6, 6, 1, 8>; };
template <> struct BShape<7, 1> { using type = FmaCfg<FEM_PRISM6, 7, 72, 6, 6, 1, 8>; };

struct BatchArgs {
  FmaArgs base;  // n = number of sorted positions, perm/offA/offb set
  const double *qp[kMaxP + 1];
  const void *phi[kMaxP + 1];
  const int4 *items;  // {(p << 4) | variant, tile index, first sorted position, end position}
  int nitems;
  unsigned *counter;  // next item (zeroed before the launch)
};

template <class T, int P, int V>
__device__ __forceinline__ void run_item(const BatchArgs &a, const int4 &it, unsigned char *smem) {
  using C = typename BShape<P, V>::type;
  fma_body<T, C>(a.base, a.qp[P], static_cast<const T *>(a.phi[P]), it.z, it.w, it.y / C::TILES,
                 it.y % C::TILES, smem);
}

// FP32 bodies are capped at 128 registers (two CTAs per SM: the FMA bodies
// need the extra warps to hide latency; measured 575 ms vs 720 ms uncapped on
// the 500k mixed mesh although the largest bodies spill a little); the FP64
// ones are bound by the FP64 pipe, so one CTA per SM costs nothing.
template <class T>
__global__ void __launch_bounds__(kBatchThreads, sizeof(T) == 4 ? 2 : 1) batch_kernel(const BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_item;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int i = s_item;
    __syncthreads();
    if (i >= a.nitems) break;
    const int4 it = a.items[i];
    switch (it.x) {
#define FEM_ITEM(P, V) \
  case (P << 4) | V: run_item<T, P, V>(a, it, smem); break;
      FEM_ITEM(1, 0) FEM_ITEM(1, 1) FEM_ITEM(2, 0) FEM_ITEM(2, 1) FEM_ITEM(3, 0) FEM_ITEM(3, 1)
      FEM_ITEM(4, 0) FEM_ITEM(4, 1) FEM_ITEM(5, 0) FEM_ITEM(5, 1) FEM_ITEM(6, 0) FEM_ITEM(6, 1)
      FEM_ITEM(7, 0) FEM_ITEM(7, 1)
#undef FEM_ITEM
      default: break;
    }
  }
}

// ---- host-side shape queries ----
struct ShapeInfo {
  int epb, tiles, nt;
  size_t smem64, smem32;
};

template <int P, int V>
static ShapeInfo shape_info_pv() {
  using C = typename BShape<P, V>::type;
  return {C::EPB, C::TILES, C::NT, C::template smem_bytes<double>(), C::template smem_bytes<float>()};
}

static ShapeInfo shape_info(int p, int v) {
  switch ((p << 4) | v) {
#define FEM_SI(P, V) \
  case (P << 4) | V: return shape_info_pv<P, V>();
    FEM_SI(1, 0) FEM_SI(1, 1) FEM_SI(2, 0) FEM_SI(2, 1) FEM_SI(3, 0) FEM_SI(3, 1) FEM_SI(4, 0)
    FEM_SI(4, 1) FEM_SI(5, 0) FEM_SI(5, 1) FEM_SI(6, 0) FEM_SI(6, 1) FEM_SI(7, 0) FEM_SI(7, 1)
#undef FEM_SI
  }
  return {0, 0, 0, 0, 0};
}

static size_t batch_smem(bool f64) {
  size_t m = 0;
  for (int p = 1; p <= kMaxP; p++)
    for (int v = 0; v < kVariants; v++) {
      ShapeInfo si = shape_info(p, v);
      m = std::max(m, f64 ? si.smem64 : si.smem32);
    }
  return m;
}

// per-degree launch of the specialised kernel over bin [k0, k0 + n) of the sorted positions
template <class T, int P, int V>
static int launch_loop_pv(FmaArgs a, void *stream) {
  using C = typename BShape<P, V>::type;
  return launch_fma_cfg<T, C>(a, stream);
}

template <class T>
static int launch_loop(int p, int v, const FmaArgs &a, void *stream) {
  if (v == kStandalone)
    return sizeof(T) == 8 ? launch_fma_f64(FEM_PRISM6, p, a, stream) : launch_fma_f32(FEM_PRISM6, p, a, stream);
  switch ((p << 4) | v) {
#define FEM_LL(P, V) \
  case (P << 4) | V: return launch_loop_pv<T, P, V>(a, stream);
    FEM_LL(1, 0) FEM_LL(1, 1) FEM_LL(2, 0) FEM_LL(2, 1) FEM_LL(3, 0) FEM_LL(3, 1) FEM_LL(4, 0)
    FEM_LL(4, 1) FEM_LL(5, 0) FEM_LL(5, 1) FEM_LL(6, 0) FEM_LL(6, 1) FEM_LL(7, 0) FEM_LL(7, 1)
#undef FEM_LL
  }
  return FEM_EINVAL;
}

}  // namespace fem

// ---------------------------------------------------------------- plan object
struct fem_plan_s {
  fem_tables t = nullptr;
  int device = 0;  // the device current at creation (the tables' device)
  int prec = 0, layout = 0, flags = 0;
  int64_t totA = 0, totb = 0;  // values of A_out and b_out
  int shrink_next = 0;         // test hook of checked builds (fem_debug_shrink_bound)
  int64_t n = 0;
  std::string cache;
  int64_t bin_off[fem::kMaxP + 2] = {0};  // sorted positions of each degree's bin
  int variant[fem::kMaxP + 1] = {0};
  bool tuned = false;
  double tuned_ms[fem::kMaxP + 1][fem::kMaxVariants] = {{0}};
  // device data (plan-owned)
  int64_t *perm = nullptr, *offA = nullptr, *offb = nullptr;
  int4 *items = nullptr;
  int nitems = 0;
  unsigned *counter = nullptr;
  std::vector<int4> h_items;
  // graph
  cudaStream_t cap = nullptr;
  cudaStream_t branch[fem::kMaxP + 1] = {nullptr};  // concurrent mode: one stream per degree
  cudaEvent_t fork = nullptr, join[fem::kMaxP + 1] = {nullptr};
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  const void *key[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int64_t key_stride = -1;
};

namespace fem {

static int plan_fail(const char *what, cudaError_t e) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return FEM_ECUDA;
}

static bool per_degree(const fem_plan_s *pl) { return (pl->flags & (FEM_PLAN_LOOP | FEM_PLAN_CONCURRENT)) != 0; }
static bool tensor_plan(const fem_plan_s *pl) { return pl->prec == FEM_BF16X3 || pl->prec == FEM_F16X3; }
// candidates of a degree's per-degree launch
static int loop_variants(const fem_plan_s *pl) { return tensor_plan(pl) ? kMaxVariants : kMaxVariants - 1; }

static double item_cost(int p) {  // relative cost of one element of degree p (contraction flops)
  const double ns = ns_of(FEM_PRISM6, p), nq = nq_of(FEM_PRISM6, p);
  return 8.0 * nq * ns * ns + 150.0 * nq;
}

// Work items of all bins (or of one bin when only_p > 0) for the given
// per-degree variants; bin_off[p] .. bin_off[p+1] are the sorted positions of
// degree p.  Appends to out (cleared first).
static void build_items_raw(const int64_t *bin_off, const int *variant, int only_p, std::vector<int4> &out) {
  out.clear();
  std::vector<std::pair<double, int4>> v;
  for (int p = 1; p <= kMaxP; p++) {
    if (only_p > 0 && p != only_p) continue;
    const int64_t k0 = bin_off[p], k1 = bin_off[p + 1];
    if (k1 <= k0) continue;
    // the persistent kernel's shapes only (a per-degree plan's uniform-degree
    // variant has no work-list form; such plans do not use the list)
    const int vp = variant[p] < kVariants ? variant[p] : 0;
    const ShapeInfo si = shape_info(p, vp);
    for (int64_t k = k0; k < k1; k += si.epb) {
      const int64_t ke = std::min<int64_t>(k + si.epb, k1);
      for (int t = 0; t < si.tiles * si.tiles; t++) {
        int4 it;
        it.x = (p << 4) | vp;
        it.y = t;
        it.z = (int)k;
        it.w = (int)ke;
        v.push_back({item_cost(p) * (double)(ke - k) / (si.tiles * si.tiles), it});
      }
    }
  }
  // most expensive items first (longest-processing-time order), stable in position
  std::stable_sort(v.begin(), v.end(), [](const std::pair<double, int4> &a, const std::pair<double, int4> &b) {
    return a.first > b.first;
  });
  for (auto &x : v) out.push_back(x.second);
}

static void build_items(const fem_plan_s *pl, int only_p, std::vector<int4> &out) {
  build_items_raw(pl->bin_off, pl->variant, only_p, out);
}

static int upload_items(fem_plan_s *pl, const std::vector<int4> &items) {
  if ((int)items.size() > pl->nitems) {
    if (pl->items) cudaFree(pl->items);
    pl->items = nullptr;
    cudaError_t e = cudaMalloc((void **)&pl->items, sizeof(int4) * std::max<size_t>(items.size(), 1));
    if (e != cudaSuccess) return plan_fail("cudaMalloc(items)", e);
  }
  pl->nitems = (int)items.size();
  if (!items.empty()) {
    cudaError_t e = cudaMemcpy(pl->items, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return plan_fail("cudaMemcpy(items)", e);
  }
  return FEM_OK;
}

static BatchArgs batch_args_raw(fem_tables t, int prec, const FmaArgs &base, const int4 *items, int nitems,
                                unsigned *counter) {
  BatchArgs b;
  b.base = base;
  for (int p = 0; p <= kMaxP; p++) {
    const DevTable &d = t->tab[p];
    b.qp[p] = d.qp;
    b.phi[p] = prec == FEM_F64 ? (const void *)d.phi64 : (const void *)d.phi32;
  }
  b.items = items;
  b.nitems = nitems;
  b.counter = counter;
  return b;
}

static BatchArgs batch_args(const fem_plan_s *pl, const FmaArgs &base) {
  return batch_args_raw(pl->t, pl->prec, base, pl->items, pl->nitems, pl->counter);
}

// Zero the work counter and launch the persistent kernel (no allocation).
static int launch_batch_raw(bool f64, const BatchArgs &b, cudaStream_t s) {
  const size_t smem = batch_smem(f64);
  cudaError_t e = cudaMemsetAsync(b.counter, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return plan_fail("cudaMemsetAsync(counter)", e);
  int dev = 0, nsm = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (f64) {
    cudaFuncSetAttribute(batch_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<double>, kBatchThreads, smem);
  } else {
    cudaFuncSetAttribute(batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<float>, kBatchThreads, smem);
  }
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)nsm * per_sm;
  if (grid > b.nitems) grid = std::max(b.nitems, 1);
  if (f64)
    batch_kernel<double><<<(unsigned)grid, kBatchThreads, smem, s>>>(b);
  else
    batch_kernel<float><<<(unsigned)grid, kBatchThreads, smem, s>>>(b);
  e = cudaGetLastError();
  if (e != cudaSuccess) return plan_fail("batch_kernel launch", e);
  return FEM_OK;
}

static int launch_batch(const fem_plan_s *pl, const BatchArgs &b, cudaStream_t s) {
  return launch_batch_raw(pl->prec == FEM_F64, b, s);
}

// One launch over the bin of degree p with variant v (per-degree modes).
static int launch_bin(const fem_plan_s *pl, int p, int v, const FmaArgs &base, cudaStream_t s) {
  const int64_t k0 = pl->bin_off[p], k1 = pl->bin_off[p + 1];
  const DevTable &d = pl->t->tab[p];
  if (v == kTensor) {
    TcLaunch l;
    l.n = k1 - k0;
    l.coords = base.coords;
    l.coeffs = base.coeffs;
    l.cstride = base.cstride;
    l.A = base.A;
    l.b = base.b;
    l.status = base.status;
    l.layout = base.layout;
    l.err = pl->t->d_err;
    l.stall = 0;
    l.perm = pl->perm + k0;
    l.offA = base.offA;
    l.offb = base.offb;
    l.limA = base.limA;
    l.limb = base.limb;
    l.nmesh = base.nmesh;
    return launch_tc(p, pl->prec == FEM_F16X3, d, l, s);
  }
  FmaArgs a = base;
  a.n = k1 - k0;
  a.perm = pl->perm + k0;
  a.qp = d.qp;
  a.phi = pl->prec == FEM_F64 ? (const void *)d.phi64 : (const void *)d.phi32;
  return pl->prec == FEM_F64 ? launch_loop<double>(p, v, a, s) : launch_loop<float>(p, v, a, s);
}

static int launch_per_p_loop(const fem_plan_s *pl, const FmaArgs &base, cudaStream_t s) {
  for (int p = 1; p <= kMaxP; p++) {
    if (pl->bin_off[p + 1] <= pl->bin_off[p]) continue;
    const int rc = launch_bin(pl, p, pl->variant[p], base, s);
    if (rc != FEM_OK) return rc;
  }
  return FEM_OK;
}

// One graph with a branch per degree: each branch runs the specialised kernel
// of its bin on its own stream, the branches overlap (enqueued inside a
// capture on pl->cap, forked and joined with events).
static int launch_concurrent(fem_plan_s *pl, const FmaArgs &base, cudaStream_t s) {
  cudaError_t e = cudaEventRecord(pl->fork, s);
  if (e != cudaSuccess) return plan_fail("cudaEventRecord(fork)", e);
  for (int p = 1; p <= kMaxP; p++) {
    const int64_t k0 = pl->bin_off[p], k1 = pl->bin_off[p + 1];
    if (k1 <= k0) continue;
    e = cudaStreamWaitEvent(pl->branch[p], pl->fork, 0);
    if (e != cudaSuccess) return plan_fail("cudaStreamWaitEvent(fork)", e);
    const int rc = launch_bin(pl, p, pl->variant[p], base, pl->branch[p]);
    if (rc != FEM_OK) return rc;
    e = cudaEventRecord(pl->join[p], pl->branch[p]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, pl->join[p], 0);
    if (e != cudaSuccess) return plan_fail("join", e);
  }
  return FEM_OK;
}

static std::string cache_key(const fem_plan_s *pl, int p) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::ostringstream o;
  o << prop.name << "|sm" << prop.major << prop.minor << "|prec" << pl->prec << "|layout" << pl->layout << "|p" << p
    << (per_degree(pl) ? "|per-degree" : "|persistent");
  std::string k = o.str();
  for (char &c : k)
    if (c == ' ') c = '_';
  return k;
}

static bool cache_lookup(const fem_plan_s *pl, int p, int *v) {
  if (pl->cache.empty()) return false;
  std::ifstream f(pl->cache);
  std::string k, key = cache_key(pl, p);
  int val;
  double ms;
  while (f >> k >> val >> ms)
    if (k == key && val >= 0 && val < (per_degree(pl) ? loop_variants(pl) : kVariants)) {
      *v = val;
      return true;
    }
  return false;
}

static void cache_store(const fem_plan_s *pl, int p) {
  if (pl->cache.empty()) return;
  std::ofstream f(pl->cache, std::ios::app);
  f << cache_key(pl, p) << " " << pl->variant[p] << " " << pl->tuned_ms[p][pl->variant[p]] << "\n";
}

// Time both candidate shapes of each degree on the plan's elements (the
// persistent kernel restricted to one bin) and keep the faster one.
static int autotune(fem_plan_s *pl, const FmaArgs &base, cudaStream_t s) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int rc = FEM_OK;
  for (int p = 1; p <= kMaxP && rc == FEM_OK; p++) {
    if (pl->bin_off[p + 1] <= pl->bin_off[p]) continue;
    int v;
    if (cache_lookup(pl, p, &v)) {
      pl->variant[p] = v;
      continue;
    }
    double best = 1e30;
    int bestv = 0;
    if (per_degree(pl)) {  // time the candidates as they are launched: one kernel over the bin
      for (int cand = 0; cand < loop_variants(pl) && rc == FEM_OK; cand++) {
        float tmin = 1e30f;
        for (int rep = 0; rep < 3 && rc == FEM_OK; rep++) {
          cudaEventRecord(e0, s);
          rc = launch_bin(pl, p, cand, base, s);
          cudaEventRecord(e1, s);
          cudaError_t err = cudaEventSynchronize(e1);
          if (err != cudaSuccess) rc = plan_fail("autotune", err);
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (rep > 0) tmin = std::min(tmin, ms);  // first run warms up
        }
        pl->tuned_ms[p][cand] = tmin;
        if (tmin < best) {
          best = tmin;
          bestv = cand;
        }
      }
      pl->variant[p] = bestv;
      cache_store(pl, p);
      continue;
    }
    for (int cand = 0; cand < kVariants && rc == FEM_OK; cand++) {
      pl->variant[p] = cand;
      std::vector<int4> items;
      build_items(pl, p, items);
      rc = upload_items(pl, items);
      if (rc != FEM_OK) break;
      BatchArgs b = batch_args(pl, base);
      float tmin = 1e30f;
      for (int rep = 0; rep < 3 && rc == FEM_OK; rep++) {
        cudaEventRecord(e0, s);
        rc = launch_batch(pl, b, s);
        cudaEventRecord(e1, s);
        cudaError_t err = cudaEventSynchronize(e1);
        if (err != cudaSuccess) rc = plan_fail("autotune", err);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) tmin = std::min(tmin, ms);  // first run warms up
      }
      pl->tuned_ms[p][cand] = tmin;
      if (tmin < best) {
        best = tmin;
        bestv = cand;
      }
    }
    pl->variant[p] = bestv;
    cache_store(pl, p);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc == FEM_OK) {
    std::vector<int4> items;
    build_items(pl, 0, items);
    rc = upload_items(pl, items);
  }
  pl->tuned = true;
  return rc;
}

static void drop_graph(fem_plan_s *pl) {
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  pl->exec = nullptr;
  pl->graph = nullptr;
}

}  // namespace fem

namespace fem {

// ---------------------------------------------------------------- allocation-free variant
//
// Some callers cannot allocate device memory: code that runs under a fixed
// memory budget or pool, inside a host that has handed all device memory to
// its own allocator, or that must not call cudaMalloc on a hot path because it
// synchronises the device.  fem_integrate_mixed_noalloc serves them: it runs
// the mixed-degree persistent kernel with all of its scratch (work counter,
// work list, degree permutation, output offsets) in the file-scope device
// array below instead of plan-owned allocations.  The array is a fixed
// kNoAllocBytes (about 1.4 MB) that every GPU which loads this library keeps
// until the process exits; it limits a call to kNoAllocMaxElems elements and
// kNoAllocMaxItems work items.
constexpr int64_t kNoAllocMaxElems = 16384;
constexpr int64_t kNoAllocMaxItems = 65536;
constexpr size_t kNoAllocOffItems = 256;  // the counter sits in the first 256 bytes
constexpr size_t kNoAllocOffPerm = kNoAllocOffItems + sizeof(int4) * kNoAllocMaxItems;
constexpr size_t kNoAllocOffA = kNoAllocOffPerm + sizeof(int64_t) * kNoAllocMaxElems;
constexpr size_t kNoAllocOffB = kNoAllocOffA + sizeof(int64_t) * kNoAllocMaxElems;
constexpr size_t kNoAllocBytes = kNoAllocOffB + sizeof(int64_t) * kNoAllocMaxElems;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
static unsigned char *g_noalloc_dev[kNoAllocMaxDevices] = {nullptr};
static std::mutex g_noalloc_mutex;  // guards the host staging arrays below
static int4 g_noalloc_h_items[kNoAllocMaxItems];
static int64_t g_noalloc_h_perm[kNoAllocMaxElems];
static int64_t g_noalloc_h_offA[kNoAllocMaxElems];
static int64_t g_noalloc_h_offb[kNoAllocMaxElems];

}  // namespace fem

using namespace fem;

extern "C" {

int fem_integrate_mixed_noalloc(fem_tables t, int64_t n_elem, const int8_t *p_host, const double *coords,
                                const double *coeffs, int64_t coeff_stride, int prec, int layout, void *A_out,
                                void *b_out, int32_t *status, void *stream) {
  if (rule_check(t, "fem_integrate_mixed_noalloc") != FEM_OK) return FEM_EUNSUPPORTED;
  if (!t || t->elem != FEM_PRISM6) {
    set_error("fem_integrate_mixed_noalloc: needs prism tables");
    return FEM_EINVAL;
  }
  if (n_elem < 0 || n_elem > kNoAllocMaxElems) {
    set_error("fem_integrate_mixed_noalloc: n_elem must be in 0..16384 (the fixed scratch size)");
    return FEM_EINVAL;
  }
  if (prec != FEM_F64 && prec != FEM_F32) {
    set_error("fem_integrate_mixed_noalloc: FP64 / FP32 only");
    return FEM_EUNSUPPORTED;
  }
  if (layout != FEM_OUT_FULL && layout != FEM_OUT_SYMPACKED) {
    set_error("fem_integrate_mixed_noalloc: unknown layout");
    return FEM_EINVAL;
  }
  if (n_elem == 0) return FEM_OK;
  if (!p_host || !coords || !coeffs || !A_out || coeff_stride < n_elem) {
    set_error("fem_integrate_mixed_noalloc: NULL buffer or coeff_stride < n_elem");
    return FEM_EINVAL;
  }
  if ((((uintptr_t)coords | (uintptr_t)coeffs) & 7) || ((uintptr_t)A_out & 15)) {
    set_error("fem_integrate_mixed_noalloc: misaligned buffer");
    return FEM_EINVAL;
  }
  int64_t bin_off[kMaxP + 2] = {0}, cur[kMaxP + 2];
  for (int64_t e = 0; e < n_elem; e++) {
    const int p = p_host[e];
    if (p < t->p_min || p > t->p_max) {
      set_error("fem_integrate_mixed_noalloc: an element's degree is not in the tables");
      return FEM_EINVAL;
    }
    bin_off[p + 1]++;
  }
  for (int p = 1; p <= kMaxP; p++) bin_off[p + 1] += bin_off[p];
  // one-time set-up per device: the device address of the scratch array
  int dev = 0;
  cudaError_t err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return plan_fail("cudaGetDevice", err);
  if (dev != t->device) {
    set_error("fem_integrate_mixed_noalloc: tables live on another device");
    return FEM_EINVAL;
  }
  if (dev < 0 || dev >= kNoAllocMaxDevices) {
    set_error("fem_integrate_mixed_noalloc: device index out of range");
    return FEM_EUNSUPPORTED;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_dev[dev]) {
    void *ptr = nullptr;
    err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (err != cudaSuccess) return plan_fail("cudaGetSymbolAddress(scratch)", err);
    g_noalloc_dev[dev] = static_cast<unsigned char *>(ptr);
  }
  unsigned char *base = g_noalloc_dev[dev];
  // host side: counting sort by degree, output offsets, work list (default shapes)
  for (int p = 0; p <= kMaxP + 1; p++) cur[p] = bin_off[p];
  for (int64_t e = 0; e < n_elem; e++) g_noalloc_h_perm[cur[p_host[e]]++] = e;
  int64_t tot[2] = {0, 0};
  int rc = fem_output_offsets(FEM_PRISM6, p_host, n_elem, layout, g_noalloc_h_offA, g_noalloc_h_offb, tot);
  if (rc != FEM_OK) return rc;
  int variant[kMaxP + 1] = {0};
  std::vector<int4> items;
  build_items_raw(bin_off, variant, 0, items);
  if ((int64_t)items.size() > kNoAllocMaxItems) {
    set_error("fem_integrate_mixed_noalloc: more than 65536 work items (reduce n_elem)");
    return FEM_EINVAL;
  }
  std::copy(items.begin(), items.end(), g_noalloc_h_items);
  cudaStream_t s = (cudaStream_t)stream;
  // pageable-source copies: each call returns once the host data is staged
  err = cudaMemcpyAsync(base + kNoAllocOffItems, g_noalloc_h_items, sizeof(int4) * items.size(),
                        cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(base + kNoAllocOffPerm, g_noalloc_h_perm, sizeof(int64_t) * n_elem,
                          cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(base + kNoAllocOffA, g_noalloc_h_offA, sizeof(int64_t) * n_elem, cudaMemcpyHostToDevice, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(base + kNoAllocOffB, g_noalloc_h_offb, sizeof(int64_t) * n_elem, cudaMemcpyHostToDevice, s);
  if (err != cudaSuccess) return plan_fail("fem_integrate_mixed_noalloc: staging copy", err);
  FmaArgs a;
  a.n = n_elem;
  a.coords = coords;
  a.coeffs = coeffs;
  a.cstride = coeff_stride;
  a.qp = nullptr;
  a.phi = nullptr;
  a.A = A_out;
  a.b = b_out;
  a.status = status;
  a.layout = layout;
  a.perm = reinterpret_cast<const int64_t *>(base + kNoAllocOffPerm);
  a.offA = reinterpret_cast<const int64_t *>(base + kNoAllocOffA);
  a.offb = reinterpret_cast<const int64_t *>(base + kNoAllocOffB);
  a.err = t->d_err;
  a.nmesh = n_elem;
  a.limA = tot[0];
  a.limb = tot[1];
  BatchArgs b = batch_args_raw(t, prec, a, reinterpret_cast<const int4 *>(base + kNoAllocOffItems),
                               (int)items.size(), reinterpret_cast<unsigned *>(base));
  return launch_batch_raw(prec == FEM_F64, b, s);  // zeroes the counter, then launches
}



int fem_output_offsets(int elem, const int8_t *p_host, int64_t n, int layout, int64_t *offA, int64_t *offb,
                       int64_t *totals) {
  if (n < 0 || (n > 0 && !p_host)) {
    set_error("fem_output_offsets: bad n or NULL degrees");
    return FEM_EINVAL;
  }
  int64_t a = 0, b = 0;
  for (int64_t e = 0; e < n; e++) {
    const int p = p_host[e];
    const int64_t m = fem_matrix_size(elem, p, layout);
    if (m < 0) {
      set_error("fem_output_offsets: degree out of range");
      return FEM_EINVAL;
    }
    if (offA) offA[e] = a;
    if (offb) offb[e] = b;
    a += m;
    b += ns_of(elem, p);
  }
  if (totals) {
    totals[0] = a;
    totals[1] = b;
  }
  return FEM_OK;
}

int fem_plan_create(fem_tables t, int64_t n_elem, const int8_t *p_host, int prec, int layout, int flags,
                    const char *tune_cache, fem_plan *out) {
  if (rule_check(t, "fem_plan_create") != FEM_OK) return FEM_EUNSUPPORTED;
  if (!out) {
    set_error("fem_plan_create: out is NULL");
    return FEM_EINVAL;
  }
  *out = nullptr;
  if (!t || t->elem != FEM_PRISM6) {
    set_error("fem_plan_create: needs prism tables");
    return FEM_EINVAL;
  }
  if (n_elem < 0 || (n_elem > 0 && !p_host) || n_elem > 0x7fffffffLL) {
    set_error("fem_plan_create: bad n_elem or NULL degrees");
    return FEM_EINVAL;
  }
  const bool tc = prec == FEM_BF16X3 || prec == FEM_F16X3;
  if (prec != FEM_F64 && prec != FEM_F32 && !tc) {
    set_error("fem_plan_create: unknown precision");
    return FEM_EUNSUPPORTED;
  }
  if (tc && !(flags & (FEM_PLAN_LOOP | FEM_PLAN_CONCURRENT))) {
    set_error("fem_plan_create: tensor-core precisions need FEM_PLAN_LOOP or FEM_PLAN_CONCURRENT");
    return FEM_EUNSUPPORTED;
  }
  if (layout != FEM_OUT_FULL && layout != FEM_OUT_SYMPACKED) {
    set_error("fem_plan_create: unknown layout");
    return FEM_EINVAL;
  }
  int dev = 0;
  cudaError_t derr = cudaGetDevice(&dev);
  if (derr != cudaSuccess) return plan_fail("cudaGetDevice", derr);
  if (dev != t->device) {
    set_error("fem_plan_create: tables live on another device");
    return FEM_EINVAL;
  }
  std::vector<int64_t> cnt(kMaxP + 2, 0);
  for (int64_t e = 0; e < n_elem; e++) {
    const int p = p_host[e];
    if (p < t->p_min || p > t->p_max) {
      set_error("fem_plan_create: an element's degree is not in the tables");
      return FEM_EINVAL;
    }
    cnt[p]++;
  }
  fem_plan pl = new (std::nothrow) fem_plan_s();
  if (!pl) return FEM_ENOMEM;
  pl->t = t;
  pl->device = dev;
  pl->prec = prec;
  pl->layout = layout;
  pl->flags = flags;
  pl->n = n_elem;
  if (tune_cache) pl->cache = tune_cache;
  pl->bin_off[1] = 0;
  for (int p = 1; p <= kMaxP; p++) pl->bin_off[p + 1] = pl->bin_off[p] + cnt[p];
  if (per_degree(pl))  // untuned per-degree launches use the uniform-degree kernels
    for (int p = 1; p <= kMaxP; p++) pl->variant[p] = tensor_plan(pl) && p >= 3 ? kTensor : kStandalone;
  // counting sort by degree (stable)
  std::vector<int64_t> perm(std::max<int64_t>(n_elem, 1)), offA(std::max<int64_t>(n_elem, 1)),
      offb(std::max<int64_t>(n_elem, 1));
  std::vector<int64_t> cur(pl->bin_off, pl->bin_off + kMaxP + 2);
  for (int64_t e = 0; e < n_elem; e++) perm[cur[p_host[e]]++] = e;
  int64_t tot[2];
  int rc = fem_output_offsets(FEM_PRISM6, p_host, n_elem, layout, offA.data(), offb.data(), tot);
  pl->totA = tot[0];
  pl->totb = tot[1];
  auto up = [&](int64_t **dst, const std::vector<int64_t> &src) -> int {
    cudaError_t e = cudaMalloc((void **)dst, sizeof(int64_t) * src.size());
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src.data(), sizeof(int64_t) * src.size(), cudaMemcpyHostToDevice);
    return e == cudaSuccess ? FEM_OK : plan_fail("plan upload", e);
  };
  if (rc == FEM_OK) rc = up(&pl->perm, perm);
  if (rc == FEM_OK) rc = up(&pl->offA, offA);
  if (rc == FEM_OK) rc = up(&pl->offb, offb);
  if (rc == FEM_OK) {
    cudaError_t e = cudaMalloc((void **)&pl->counter, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess && (flags & FEM_PLAN_CONCURRENT)) {
      e = cudaEventCreateWithFlags(&pl->fork, cudaEventDisableTiming);
      for (int p = 1; p <= kMaxP && e == cudaSuccess; p++) {
        e = cudaStreamCreateWithFlags(&pl->branch[p], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->join[p], cudaEventDisableTiming);
      }
    }
    if (e != cudaSuccess) rc = plan_fail("plan setup", e);
  }
  if (rc == FEM_OK) {
    std::vector<int4> items;
    build_items(pl, 0, items);
    rc = upload_items(pl, items);
  }
  if (rc != FEM_OK) {
    fem_plan_destroy(pl);
    return rc;
  }
  *out = pl;
  return FEM_OK;
}

int fem_plan_execute(fem_plan pl, const double *coords, const double *coeffs, int64_t coeff_stride, void *A_out,
                     void *b_out, int32_t *status, void *stream) {
  if (!pl) {
    set_error("fem_plan_execute: plan is NULL");
    return FEM_EINVAL;
  }
  if (pl->n == 0) return FEM_OK;
  int dev = 0;
  cudaError_t derr = cudaGetDevice(&dev);
  if (derr != cudaSuccess) return plan_fail("cudaGetDevice", derr);
  if (dev != pl->device) {
    set_error("fem_plan_execute: the plan lives on another device");
    return FEM_EINVAL;
  }
  if (!coords || !coeffs || !A_out || coeff_stride < pl->n) {
    set_error("fem_plan_execute: NULL buffer or coeff_stride < n_elem");
    return FEM_EINVAL;
  }
  if ((((uintptr_t)coords | (uintptr_t)coeffs) & 7) || ((uintptr_t)A_out & 15)) {
    set_error("fem_plan_execute: misaligned buffer");
    return FEM_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  FmaArgs base;
  base.n = pl->n;
  base.coords = coords;
  base.coeffs = coeffs;
  base.cstride = coeff_stride;
  base.qp = nullptr;
  base.phi = nullptr;
  base.A = A_out;
  base.b = b_out;
  base.status = status;
  base.layout = pl->layout;
  base.perm = pl->perm;
  base.offA = pl->offA;
  base.offb = pl->offb;
  // checked builds: element ids and output offsets against the plan's extents
  base.err = pl->t->d_err;
  base.nmesh = pl->n;
  base.limA = pl->totA;
  base.limb = pl->totb;
  int rc = FEM_OK;
  if (pl->shrink_next) {
    // test hook of checked builds: A_out taken as one value shorter than it
    // is, so the block that ends there is refused by the checks; a direct
    // launch (no graph), the next execution is normal again
    pl->shrink_next = 0;
    base.limA = pl->totA - 1;
    if (pl->flags & FEM_PLAN_LOOP) return launch_per_p_loop(pl, base, s);
    if (pl->flags & FEM_PLAN_CONCURRENT) return launch_concurrent(pl, base, s);
    return launch_batch(pl, batch_args(pl, base), s);
  }
  if ((pl->flags & FEM_PLAN_AUTOTUNE) && !pl->tuned) {
    rc = autotune(pl, base, s);
    if (rc != FEM_OK) return rc;
    drop_graph(pl);
  }
  if (pl->flags & FEM_PLAN_LOOP) return launch_per_p_loop(pl, base, s);
  BatchArgs b = batch_args(pl, base);
  const bool conc = (pl->flags & FEM_PLAN_CONCURRENT) != 0;
  if (pl->flags & FEM_PLAN_NOGRAPH) return conc ? launch_concurrent(pl, base, s) : launch_batch(pl, b, s);
  const void *key[6] = {coords, coeffs, A_out, b_out, status, nullptr};
  bool same = pl->exec && pl->key_stride == coeff_stride;
  for (int i = 0; i < 6 && same; i++) same = key[i] == pl->key[i];
  if (!same) {
    drop_graph(pl);
    cudaError_t e = cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return plan_fail("cudaStreamBeginCapture", e);
    rc = conc ? launch_concurrent(pl, base, pl->cap) : launch_batch(pl, b, pl->cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(pl->cap, &g);
    if (rc != FEM_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return plan_fail("cudaStreamEndCapture", e);
    pl->graph = g;
    e = cudaGraphInstantiate(&pl->exec, g, 0);
    if (e != cudaSuccess) {
      drop_graph(pl);
      return plan_fail("cudaGraphInstantiate", e);
    }
    for (int i = 0; i < 6; i++) pl->key[i] = key[i];
    pl->key_stride = coeff_stride;
  }
  cudaError_t e = cudaGraphLaunch(pl->exec, s);
  if (e != cudaSuccess) return plan_fail("cudaGraphLaunch", e);
  return FEM_OK;
}

int fem_debug_shrink_bound(fem_plan pl) {
  if (!pl) {
    set_error("fem_debug_shrink_bound: plan is NULL");
    return FEM_EINVAL;
  }
  if (!kChecked) {
    set_error("fem_debug_shrink_bound: a hook of the checked build (libfem_gb300_checked.so)");
    return FEM_EUNSUPPORTED;
  }
  pl->shrink_next = 1;
  return FEM_OK;
}

int fem_plan_variant(fem_plan pl, int p, double *ms) {
  if (!pl || p < 1 || p > kMaxP) return -1;
  if (ms)
    for (int v = 0; v < kMaxVariants; v++) ms[v] = pl->tuned_ms[p][v];
  return pl->variant[p];
}

int fem_plan_destroy(fem_plan pl) {
  if (!pl) return FEM_OK;
  drop_graph(pl);
  if (pl->perm) cudaFree(pl->perm);
  if (pl->offA) cudaFree(pl->offA);
  if (pl->offb) cudaFree(pl->offb);
  if (pl->items) cudaFree(pl->items);
  if (pl->counter) cudaFree(pl->counter);
  if (pl->cap) cudaStreamDestroy(pl->cap);
  for (int p = 0; p <= kMaxP; p++) {
    if (pl->branch[p]) cudaStreamDestroy(pl->branch[p]);
    if (pl->join[p]) cudaEventDestroy(pl->join[p]);
  }
  if (pl->fork) cudaEventDestroy(pl->fork);
  delete pl;
  return FEM_OK;
}

}  // extern "C"

namespace fem {

// fem_integrate with per-element degrees (the host's classification of the
// elements by degree, Section 4.2): the tables keep one per-degree
// concurrent plan and rebuild it when the degrees, precision or layout of a
// call differ from the ones it was made for.
int integrate_mixed_cached(fem_tables t, int64_t n, const int8_t *p_host, const double *coords,
                           const double *coeffs, int64_t cstride, int prec, int layout, void *A, void *b,
                           int32_t *status, void *stream) {
  if (n < 0) {
    set_error("fem_integrate: n_elem < 0");
    return FEM_EINVAL;
  }
  if (n == 0) return FEM_OK;
  std::lock_guard<std::mutex> lock(t->mixed_mutex);
  const bool same = t->mixed && t->mixed_prec == prec && t->mixed_layout == layout &&
                    (int64_t)t->mixed_p.size() == n && std::memcmp(t->mixed_p.data(), p_host, (size_t)n) == 0;
  if (!same) {
    if (t->mixed) fem_plan_destroy(t->mixed);
    t->mixed = nullptr;
    t->mixed_p.clear();
    fem_plan pl = nullptr;
    const int rc = fem_plan_create(t, n, p_host, prec, layout, FEM_PLAN_CONCURRENT, nullptr, &pl);
    if (rc != FEM_OK) return rc;
    t->mixed = pl;
    t->mixed_p.assign(p_host, p_host + n);
    t->mixed_prec = prec;
    t->mixed_layout = layout;
  }
  return fem_plan_execute(t->mixed, coords, coeffs, cstride, A, b, status, stream);
}

}  // namespace fem
