// batch.cu - many grids advanced together: one persistent launch per step.
//
// A batch gathers contexts that were created and bound one by one (uneven
// grids, rates, time steps and boundaries; one precision, one stream).  A
// device table holds every instance's tensor maps, buffers, layout and
// coefficient block; a tile list holds (instance, strip, row segment).  Per
// time step one launch walks the tile list with a persistent grid (the
// FP32 kernel's CTAs claim tiles one at a time from a counter, the list
// sorted longest first, which balanced the uneven tiles 5% better than a
// fixed assignment; the FP64 kernel's CTA b takes tiles b, b + G, ...),
// copying each tile's coefficient block into shared
// memory and marching it with the same device code as the single-grid
// kernel; instances with walls get one batched wall launch before it.  The
// time loop runs as CUDA graphs of a fixed number of steps, captured once
// per starting buffer parity.  The tile shape (strip width, segment length)
// comes from mrtlb_batch_tune: timed trials, results cached on disk.
#include <cuda.h>

#include <algorithm>
#include <cstddef>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.h"
#include "march.cuh"
#include "march_pair.cuh"

namespace mrtlb {
namespace {

template <typename R>
struct BatchInst {
  CUtensorMap map[2];  // read maps of the two state buffers
  R* f[2];
  Layout L;
  Coef<R> c;
};

struct WallInst {
  Layout L;
  Coef<float> c32;   // the coefficients of the instance in both precisions
  Coef<double> c64;
  Walls w;
  void* f[2];
  int first;  // index of this instance's first wall node in the flat enumeration
};

template <typename R, int BX, int NSLOT>
__host__ __device__ constexpr size_t batch_coef_off() {
  return (Smem<R, BX, NSLOT>::bytes + 127) & ~(size_t)127;
}
template <typename R, int BX, int NSLOT>
__host__ __device__ constexpr size_t batch_smem() {
  return batch_coef_off<R, BX, NSLOT>() + sizeof(Coef<R>);
}

template <typename R, int BX, int NSLOT, int MINB>
__global__ void __launch_bounds__(BX, MINB) step_batched_kernel(const BatchInst<R>* __restrict__ insts,
                                                                const int4* __restrict__ tiles, int ntiles,
                                                                int cur, int* err) {
  using SM = Smem<R, BX, NSLOT>;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  Coef<R>* cs = reinterpret_cast<Coef<R>*>(smem_raw + batch_coef_off<R, BX, NSLOT>());
  March<R, BX, NSLOT> m;
  m.slots = reinterpret_cast<R*>(smem_raw);
  m.U = reinterpret_cast<R*>(smem_raw + SM::u_off);
  m.bars = reinterpret_cast<uint64_t*>(smem_raw + SM::bar_off);
  m.err = err;
  m.t = threadIdx.x;
  m.kbase = 0;
  if (m.t == 0) {
    for (int s = 0; s < NSLOT; ++s) mbar_init(&m.bars[s], 1);
    mbar_fence_init();
  }
  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const int4 tl = tiles[ti];  // (instance, x0, ja, jb)
    const BatchInst<R>* in = insts + tl.x;
    {
      const uint32_t* src = reinterpret_cast<const uint32_t*>(&in->c);
      uint32_t* dst = reinterpret_cast<uint32_t*>(cs);
      for (int k = m.t; k < (int)(sizeof(Coef<R>) / 4); k += BX) dst[k] = src[k];
    }
    m.L = in->L;
    m.plane = m.L.plane;
    m.map = &in->map[cur];
    m.fout = in->f[cur ^ 1];
    __syncthreads();  // coefficients in place (and the previous tile done with them)
    if (m.segment(*cs, tl.y, tl.z, tl.w)) {
      if (m.t == 0) atomicOr(err, ERRBIT_TIMEOUT);
      m.drain();
      return;
    }
    __syncthreads();
  }
}

#ifndef MRTLB_BATCH_PREFETCH
#define MRTLB_BATCH_PREFETCH 1
#endif

// FP32 with two nodes per thread (march_pair.cuh): BX/2 threads per CTA;
// each tile's coefficients are expanded into pairs as they are copied.
template <int BX, int NSLOT>
__host__ __device__ constexpr size_t batch_pair_coef_off() {
  return (PairSmem<BX, NSLOT>::bytes + 127) & ~(size_t)127;
}
template <int BX, int NSLOT>
__host__ __device__ constexpr size_t batch_pair_smem() {
  return batch_pair_coef_off<BX, NSLOT>() + sizeof(Coef<P2>);
}

template <int BX, int NSLOT, int MINB>
__global__ void __launch_bounds__(BX / 2, MINB)
    step_batched_pair_kernel(const BatchInst<float>* __restrict__ insts, const int4* __restrict__ tiles,
                             int ntiles, int cur, int* err, int* claim) {
  using SM = PairSmem<BX, NSLOT>;
  constexpr int NT = BX / 2;
  constexpr int NF = (int)(offsetof(Coef<float>, version) / sizeof(float));  // float fields
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ int next_tile;
  Coef<P2>* cs = reinterpret_cast<Coef<P2>*>(smem_raw + batch_pair_coef_off<BX, NSLOT>());
  PairMarch<BX, NSLOT> m;
  m.slots = reinterpret_cast<float*>(smem_raw);
  m.U = reinterpret_cast<float*>(smem_raw + SM::u_off);
  m.bars = reinterpret_cast<uint64_t*>(smem_raw + SM::bar_off);
  m.err = err;
  m.t = threadIdx.x;
  m.kbase = 0;
  if (m.t == 0) {
    for (int s = 0; s < NSLOT; ++s) mbar_init(&m.bars[s], 1);
    mbar_fence_init();
    // Tiles are claimed from claim[cur]; this launch clears claim[cur ^ 1]
    // for the next step (the launch before it, which used that counter, has
    // completed: launches on one stream run in order).
    if (blockIdx.x == 0) claim[cur ^ 1] = 0;
    next_tile = atomicAdd(&claim[cur], 1);
  }
  __syncthreads();
  int ti = next_tile;
  __syncthreads();  // read before thread 0 claims the next one
  while (ti < ntiles) {
    if (m.t == 0) next_tile = atomicAdd(&claim[cur], 1);  // the tile after this one
    const int4 tl = tiles[ti];  // (instance, x0, ja, jb)
    const BatchInst<float>* in = insts + tl.x;
    {
      const float* src = &in->c.a1x;
      P2* dst = &cs->a1x;
      for (int k = m.t; k < NF; k += NT) dst[k] = P2(src[k]);
      if (m.t == 0) {
        cs->version = in->c.version;
        cs->modified = in->c.modified;
      }
    }
    m.L = in->L;
    m.plane = m.L.plane;
    m.map = &in->map[cur];
    m.fout = in->f[cur ^ 1];
    __syncthreads();  // coefficients in place (and the previous tile done with them); next_tile set
    const int nti = next_tile;
    if (MRTLB_BATCH_PREFETCH && nti < ntiles) {  // the next tile streams in behind this one
      const int4 nt = tiles[nti];
      const BatchInst<float>* nin = insts + nt.x;
      m.set_next(&nin->map[cur], nin->L.xoff + nt.y - SM::HL, nt.z, nt.w);
    }
    if (m.segment(*cs, tl.y, tl.z, tl.w)) {
      if (m.t == 0) atomicOr(err, ERRBIT_TIMEOUT);
      m.drain();
      return;
    }
    m.advance();
    __syncthreads();  // (every thread has read next_tile before it is claimed again)
    ti = nti;
  }
}

template <typename R>
__global__ void walls_batched_kernel(const WallInst* __restrict__ wi, int nw, int total, int cur) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= total) return;
  int lo = 0, hi = nw - 1;  // last instance whose first wall node is <= g
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (wi[mid].first <= g) lo = mid;
    else hi = mid - 1;
  }
  const WallInst& w = wi[lo];
  const Coef<R>& c = *reinterpret_cast<const Coef<R>*>(sizeof(R) == 4 ? (const void*)&w.c32 : (const void*)&w.c64);
  wall_node<R>(reinterpret_cast<R*>(w.f[cur]), w.L, c, w.w, g - w.first);
}

// kernel variants by strip width
template <typename R> struct BatchShapes;
template <> struct BatchShapes<float> {
  static constexpr int NS = 4;
};
template <> struct BatchShapes<double> {
  static constexpr int NS = 4;
};

#ifndef MRTLB_PAIR
#define MRTLB_PAIR 1
#endif

// The dynamic shared memory the batched kernel of this shape needs, allowed
// for it in the current context (set by set_tiles, so once per batch and
// tile shape, on the batch's device, outside any stream capture).
template <typename R, int BX, int MINB>
cudaError_t allow_batched_smem() {
  constexpr int NS = BatchShapes<R>::NS;
  const auto A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if constexpr (sizeof(R) == 4 && MRTLB_PAIR)
    return cudaFuncSetAttribute(step_batched_pair_kernel<BX, NS, MINB>, A, (int)batch_pair_smem<BX, NS>());
  else
    return cudaFuncSetAttribute(step_batched_kernel<R, BX, NS, MINB>, A, (int)batch_smem<R, BX, NS>());
}

template <typename R, int BX, int MINB>
void launch_batched_bx(const void* insts, const int4* tiles, int ntiles, int grid, int cur, int* err, int* claim,
                       cudaStream_t st) {
  constexpr int NS = BatchShapes<R>::NS;
  if constexpr (sizeof(R) == 4 && MRTLB_PAIR) {
    step_batched_pair_kernel<BX, NS, MINB><<<grid, BX / 2, batch_pair_smem<BX, NS>(), st>>>(
        (const BatchInst<float>*)insts, tiles, ntiles, cur, err, claim);
  } else {
    step_batched_kernel<R, BX, NS, MINB><<<grid, BX, batch_smem<R, BX, NS>(), st>>>(
        (const BatchInst<R>*)insts, tiles, ntiles, cur, err);
  }
}

}  // namespace
}  // namespace mrtlb

struct mrtlb_batch {
  std::vector<mrtlb_ctx*> ctx;
  std::vector<void*> bufs;     // each instance's two state buffers as the tables hold them
  std::vector<double> rates;   // each instance's s[16] as the tables' coefficient blocks hold them
  int prec = MRTLB_FP32;
  cudaStream_t stream = nullptr;
  cudaStream_t cap = nullptr;  // capture stream (the legacy stream cannot be captured)
  void* d_insts = nullptr;
  WallInst* d_walls = nullptr;
  int nwall_inst = 0, total_walls = 0;
  int4* d_tiles = nullptr;
  int ntiles = 0, tiles_cap = 0;
  int bx = 0, seglen = 0, grid = 0;
  int cur = 0;
  int* err = nullptr;
  int* claim = nullptr;  // tile counters of the persistent step, one per buffer parity
  int graph_steps = 64;
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  long long nodes = 0;
  std::string last_error;
};

namespace {

int bfail(mrtlb_batch* b, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (b) b->last_error = buf;
  return code;
}

#define BCK(call, what)                                                                       \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) return bfail(b, MRTLB_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e_)); \
  } while (0)

#ifndef MRTLB_BATCH_MINB64
#define MRTLB_BATCH_MINB64 8
#endif
#ifndef MRTLB_BATCH_MINB128
#define MRTLB_BATCH_MINB128 4
#endif

int resident_per_sm(int prec, int bx) {
  if (prec == MRTLB_FP64) return 3;
  return bx == 64 ? MRTLB_BATCH_MINB64 : MRTLB_BATCH_MINB128;
}

bool shape_supported(int prec, int bx) {
  if (prec == MRTLB_FP64) return bx == 64;
  return bx == 64 || bx == 128;
}

// Instance table for strip width bx (the tensor-map box depends on it).
template <typename R>
int upload_instances(mrtlb_batch* b, int bx, const Coef<R>& (*coef)(const mrtlb_ctx*)) {
  const int n = (int)b->ctx.size();
  std::vector<BatchInst<R>> t(n);
  for (int i = 0; i < n; ++i) {
    mrtlb_ctx* c = b->ctx[i];
    if (encode_row_maps(c->L, (int)sizeof(R), c->f[0], c->f[1], bx, t[i].map))
      return bfail(b, MRTLB_ERR_CUDA, "tensor-map encoding failed for instance %d", i);
    t[i].f[0] = (R*)c->f[0];
    t[i].f[1] = (R*)c->f[1];
    t[i].L = c->L;
    t[i].c = coef(c);
  }
  if (!b->d_insts) BCK(cudaMalloc(&b->d_insts, n * sizeof(t[0])), "cudaMalloc(instance table)");
  BCK(cudaMemcpy(b->d_insts, t.data(), n * sizeof(t[0]), cudaMemcpyHostToDevice), "copy instance table");
  return MRTLB_OK;
}
const Coef<float>& coef32(const mrtlb_ctx* c) { return c->c32; }
const Coef<double>& coef64(const mrtlb_ctx* c) { return c->c64; }

void drop_graphs(mrtlb_batch* b) {
  for (int p = 0; p < 2; ++p)
    if (b->graph[p]) {
      cudaGraphExecDestroy(b->graph[p]);
      b->graph[p] = nullptr;
    }
}

int set_tiles(mrtlb_batch* b, int bx, int seglen) {
  if (!shape_supported(b->prec, bx)) return bfail(b, MRTLB_ERR_ARG, "strip width %d not available", bx);
  if (seglen < 1) return bfail(b, MRTLB_ERR_ARG, "segment length %d", seglen);
  {
    const cudaError_t e = (b->prec == MRTLB_FP64) ? allow_batched_smem<double, 64, 3>()
                          : (bx == 64)            ? allow_batched_smem<float, 64, MRTLB_BATCH_MINB64>()
                                                  : allow_batched_smem<float, 128, MRTLB_BATCH_MINB128>();
    if (e != cudaSuccess) return bfail(b, MRTLB_ERR_CUDA, "shared-memory attribute: %s", cudaGetErrorString(e));
  }
  if (bx != b->bx) {
    cudaStreamSynchronize(b->stream);  // the table may be in use by queued steps
    const int rc = (b->prec == MRTLB_FP64) ? upload_instances<double>(b, bx, coef64)
                                           : upload_instances<float>(b, bx, coef32);
    if (rc) return rc;
  }
  std::vector<int4> tiles;
  for (int i = 0; i < (int)b->ctx.size(); ++i) {
    const Layout& L = b->ctx[i]->L;
    const int nstrips = (L.i1 + bx - 1) / bx;
    for (int s = 0; s < nstrips; ++s) {
      if ((s + 1) * bx <= L.i0) continue;  // no advanced column in this strip
      for (int j = L.j0; j < L.j1; j += seglen) tiles.push_back(make_int4(i, s * bx, j, std::min(j + seglen, L.j1)));
    }
  }
  // longest segments first, so that round-robin over the persistent grid balances
  std::stable_sort(tiles.begin(), tiles.end(), [](const int4& a, const int4& c) { return (a.w - a.z) > (c.w - c.z); });
  if (b->d_tiles) cudaStreamSynchronize(b->stream);
  if ((int)tiles.size() > b->tiles_cap) {
    if (b->d_tiles) cudaFree(b->d_tiles);
    b->d_tiles = nullptr;
    BCK(cudaMalloc((void**)&b->d_tiles, tiles.size() * sizeof(int4)), "cudaMalloc(tiles)");
    b->tiles_cap = (int)tiles.size();
  }
  BCK(cudaMemcpy(b->d_tiles, tiles.data(), tiles.size() * sizeof(int4), cudaMemcpyHostToDevice), "copy tiles");
  b->ntiles = (int)tiles.size();
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (nsm <= 0) nsm = 152;
  b->grid = std::min(b->ntiles, nsm * resident_per_sm(b->prec, bx));
  if (b->grid < 1) b->grid = 1;
  b->bx = bx;
  b->seglen = seglen;
  drop_graphs(b);
  // both tile counters start at zero whatever parity the next step has (the
  // tuner's trial launches, and any launches of the old tiles, leave the
  // counter of their last parity at the old tile count)
  if (b->claim) BCK(cudaMemsetAsync(b->claim, 0, 2 * sizeof(int), b->stream), "clear tile counters");
  return MRTLB_OK;
}

// Wall table: one entry per instance with walls (its layout, coefficient
// blocks, wall data and buffers) and the running count of its wall nodes.
// Allocated on the first call; later calls rewrite it in place.
int upload_walls(mrtlb_batch* b) {
  std::vector<WallInst> w;
  int first = 0;
  for (int i = 0; i < (int)b->ctx.size(); ++i) {
    const int nwall = wall_count(b->ctx[i]->L);
    if (nwall == 0) continue;
    WallInst e;
    std::memset(&e, 0, sizeof(e));
    e.L = b->ctx[i]->L;
    e.c32 = b->ctx[i]->c32;
    e.c64 = b->ctx[i]->c64;
    e.w = b->ctx[i]->walls;
    e.f[0] = b->ctx[i]->f[0];
    e.f[1] = b->ctx[i]->f[1];
    e.first = first;
    first += nwall;
    w.push_back(e);
  }
  b->nwall_inst = (int)w.size();
  b->total_walls = first;
  if (w.empty()) return MRTLB_OK;
  if (!b->d_walls) BCK(cudaMalloc((void**)&b->d_walls, w.size() * sizeof(WallInst)), "cudaMalloc(wall table)");
  BCK(cudaMemcpy(b->d_walls, w.data(), w.size() * sizeof(WallInst), cudaMemcpyHostToDevice), "copy wall table");
  return MRTLB_OK;
}

void snapshot_rates(mrtlb_batch* b) {
  b->rates.resize(16 * b->ctx.size());
  for (size_t i = 0; i < b->ctx.size(); ++i) std::memcpy(&b->rates[16 * i], b->ctx[i]->s, 16 * sizeof(double));
}

// Rates set on an instance (mrtlb_set_rates) after its coefficient blocks
// were copied into the tables: copy them again, in place (the captured
// time loops read the tables when they run, so they stay valid).
int refresh_coefficients(mrtlb_batch* b) {
  bool changed = false;
  for (size_t i = 0; i < b->ctx.size() && !changed; ++i)
    changed = std::memcmp(&b->rates[16 * i], b->ctx[i]->s, 16 * sizeof(double)) != 0;
  if (!changed) return MRTLB_OK;
  BCK(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");  // queued steps read the old blocks
  int rc = (b->prec == MRTLB_FP64) ? upload_instances<double>(b, b->bx, coef64)
                                   : upload_instances<float>(b, b->bx, coef32);
  if (!rc) rc = upload_walls(b);
  if (rc) return rc;
  snapshot_rates(b);
  return MRTLB_OK;
}

void enqueue_batch_step(mrtlb_batch* b, int cur, cudaStream_t st) {
  if (b->total_walls > 0) {
    const int nb = (b->total_walls + 127) / 128;
    if (b->prec == MRTLB_FP64) walls_batched_kernel<double><<<nb, 128, 0, st>>>(b->d_walls, b->nwall_inst, b->total_walls, cur);
    else walls_batched_kernel<float><<<nb, 128, 0, st>>>(b->d_walls, b->nwall_inst, b->total_walls, cur);
  }
  if (b->ntiles == 0) return;
  if (b->prec == MRTLB_FP64) {
    launch_batched_bx<double, 64, 3>(b->d_insts, b->d_tiles, b->ntiles, b->grid, cur, b->err, b->claim, st);
  } else if (b->bx == 64) {
    launch_batched_bx<float, 64, MRTLB_BATCH_MINB64>(b->d_insts, b->d_tiles, b->ntiles, b->grid, cur, b->err, b->claim, st);
  } else {
    launch_batched_bx<float, 128, MRTLB_BATCH_MINB128>(b->d_insts, b->d_tiles, b->ntiles, b->grid, cur, b->err, b->claim, st);
  }
}

int ensure_graph(mrtlb_batch* b, int parity) {
  if (b->graph[parity]) return MRTLB_OK;
  BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  int cur = parity;
  for (int k = 0; k < b->graph_steps; ++k) {
    enqueue_batch_step(b, cur, b->cap);
    cur ^= 1;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
  if (e != cudaSuccess) return bfail(b, MRTLB_ERR_CUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(e));
  const cudaError_t e2 = cudaGraphInstantiate(&b->graph[parity], g, 0);
  cudaGraphDestroy(g);
  if (e2 != cudaSuccess) return bfail(b, MRTLB_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e2));
  return MRTLB_OK;
}

int run_steps(mrtlb_batch* b, long nsteps) {
  long k = 0;
  while (k < nsteps) {
    if (b->graph_steps > 0 && nsteps - k >= b->graph_steps) {
      const int rc = ensure_graph(b, b->cur);
      if (rc) return rc;
      BCK(cudaGraphLaunch(b->graph[b->cur], b->stream), "cudaGraphLaunch");
      k += b->graph_steps;
      if (b->graph_steps & 1) b->cur ^= 1;
    } else {
      enqueue_batch_step(b, b->cur, b->stream);
      b->cur ^= 1;
      ++k;
    }
  }
  BCK(cudaGetLastError(), "batched step launch");
  for (mrtlb_ctx* c : b->ctx) {
    c->cur = b->cur;
    c->steps += nsteps;
    if (nsteps > 0) ++c->gen;
  }
  return MRTLB_OK;
}

uint64_t fnv1a(const std::string& s) {
  uint64_t h = 1469598103934665603ull;
  for (unsigned char ch : s) {
    h ^= ch;
    h *= 1099511628211ull;
  }
  return h;
}

std::string signature(const mrtlb_batch* b) {
  std::string s = b->prec == MRTLB_FP64 ? "fp64" : "fp32";
  char buf[96];
  for (const mrtlb_ctx* c : b->ctx) {
    snprintf(buf, sizeof(buf), ";%dx%d:%d%d%d%d", c->L.nx, c->L.ny, c->L.bc[0], c->L.bc[1], c->L.bc[2], c->L.bc[3]);
    s += buf;
  }
  int dev = 0;
  cudaDeviceProp prop;
  cudaGetDevice(&dev);
  if (cudaGetDeviceProperties(&prop, dev) == cudaSuccess) s += std::string(";") + prop.name;
  snprintf(buf, sizeof(buf), "%016llx", (unsigned long long)fnv1a(s));
  return buf;
}

}  // namespace

extern "C" int mrtlb_batch_create(mrtlb_ctx* const* ctxs, int n, mrtlb_batch** out) {
  if (!out) return MRTLB_ERR_ARG;
  *out = nullptr;
  if (!ctxs || n < 1) return MRTLB_ERR_ARG;
  mrtlb_batch* b = new mrtlb_batch();
  for (int i = 0; i < n; ++i) {
    mrtlb_ctx* c = ctxs[i];
    if (!c || !c->f[0] || !c->f[1] || !c->plan.ok) {
      delete b;
      return MRTLB_ERR_STATE;
    }
    if (i > 0 && (c->prec != ctxs[0]->prec || c->stream != ctxs[0]->stream || c->cur != ctxs[0]->cur)) {
      delete b;
      return MRTLB_ERR_ARG;
    }
    b->ctx.push_back(c);
    b->bufs.push_back(c->f[0]);
    b->bufs.push_back(c->f[1]);
    b->nodes += (long long)c->L.nx * c->L.ny;
  }
  b->prec = ctxs[0]->prec;
  b->stream = ctxs[0]->stream;
  b->cur = ctxs[0]->cur;
  auto cleanup = [&](int rc) {
    mrtlb_batch_destroy(b);
    return rc;
  };
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) return cleanup(MRTLB_ERR_CUDA);
  if (cudaMalloc((void**)&b->err, 256) != cudaSuccess || cudaMemset(b->err, 0, 256) != cudaSuccess)
    return cleanup(MRTLB_ERR_CUDA);
  if (cudaMalloc((void**)&b->claim, 2 * sizeof(int)) != cudaSuccess ||
      cudaMemset(b->claim, 0, 2 * sizeof(int)) != cudaSuccess)
    return cleanup(MRTLB_ERR_CUDA);
  int rc = upload_walls(b);
  if (rc) return cleanup(rc);
  rc = set_tiles(b, b->prec == MRTLB_FP64 ? 64 : 128, 32);
  if (rc) return cleanup(rc);
  snapshot_rates(b);
  *out = b;
  return MRTLB_OK;
}

extern "C" int mrtlb_batch_set_tiles(mrtlb_batch* b, int bx, int seglen) {
  if (!b) return MRTLB_ERR_ARG;
  return set_tiles(b, bx, seglen);
}

extern "C" int mrtlb_batch_get_tiles(const mrtlb_batch* b, int* bx, int* seglen, int* ntiles, int* grid) {
  if (!b) return MRTLB_ERR_ARG;
  if (bx) *bx = b->bx;
  if (seglen) *seglen = b->seglen;
  if (ntiles) *ntiles = b->ntiles;
  if (grid) *grid = b->grid;
  return MRTLB_OK;
}

extern "C" int mrtlb_batch_set_graph_steps(mrtlb_batch* b, int steps) {
  if (!b || steps < 0) return MRTLB_ERR_ARG;
  drop_graphs(b);
  b->graph_steps = steps;
  return MRTLB_OK;
}

extern "C" int mrtlb_batch_step(mrtlb_batch* b, long nsteps) {
  TraceRange trace_("mrtlb_batch_step");
  if (!b || nsteps < 0) return MRTLB_ERR_ARG;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    const mrtlb_ctx* c = b->ctx[i];
    if (c->f[0] != b->bufs[2 * i] || c->f[1] != b->bufs[2 * i + 1])
      return bfail(b, MRTLB_ERR_STATE, "instance %d was bound to other buffers after the batch was made", (int)i);
    if (c->cur != b->cur) return bfail(b, MRTLB_ERR_STATE, "an instance was stepped or reset outside the batch");
  }
  const int rc = refresh_coefficients(b);
  if (rc) return rc;
  return run_steps(b, nsteps);
}

extern "C" int mrtlb_batch_sync(mrtlb_batch* b) {
  if (!b) return MRTLB_ERR_ARG;
  int h = 0;
  BCK(cudaMemcpyAsync(&h, b->err, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "read error word");
  BCK(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  if (h & ERRBIT_TIMEOUT) return bfail(b, MRTLB_ERR_TIMEOUT, "a bounded device-side wait gave up");
  if (h & ERRBIT_NONPHYSICAL) return bfail(b, MRTLB_ERR_NONPHYSICAL, "non-physical state met by a batched step");
  return MRTLB_OK;
}

extern "C" long long mrtlb_batch_nodes(const mrtlb_batch* b) { return b ? b->nodes : -1; }

extern "C" int mrtlb_batch_tune(mrtlb_batch* b, const char* cache_path, int trial_steps, int* bx_out,
                                int* seglen_out) {
  if (!b) return MRTLB_ERR_ARG;
  if (trial_steps < 1) trial_steps = 8;
  {
    const int rc = refresh_coefficients(b);  // (the trials step with the instances' current rates)
    if (rc) return rc;
  }
  const std::string sig = signature(b);
  // cached?
  if (cache_path && cache_path[0]) {
    if (FILE* fh = fopen(cache_path, "r")) {
      char key[64];
      int bx = 0, sl = 0;
      double us = 0;
      int found = 0;
      while (fscanf(fh, "%63s %d %d %lf", key, &bx, &sl, &us) == 4)
        if (sig == key && shape_supported(b->prec, bx)) {
          found = 1;
          break;
        }
      fclose(fh);
      if (found) {
        const int rc = set_tiles(b, bx, sl);
        if (rc) return rc;
        if (bx_out) *bx_out = bx;
        if (seglen_out) *seglen_out = sl;
        return MRTLB_OK;
      }
    }
  }
  // save the states so that the trials leave them untouched
  BCK(cudaStreamSynchronize(b->stream), "cudaStreamSynchronize");
  std::vector<void*> saved(b->ctx.size(), nullptr);
  const int cur0 = b->cur;
  auto release = [&]() {
    for (void* p : saved)
      if (p) cudaFree(p);
  };
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    if (cudaMalloc(&saved[i], b->ctx[i]->state_bytes) != cudaSuccess) {
      release();
      return bfail(b, MRTLB_ERR_CUDA, "cudaMalloc(tuning snapshot)");
    }
    cudaMemcpyAsync(saved[i], b->ctx[i]->f[cur0], b->ctx[i]->state_bytes, cudaMemcpyDeviceToDevice, b->stream);
  }
  const int graph_steps = b->graph_steps;
  b->graph_steps = 0;  // time plain launches
  const int bxs[2] = {64, 128};
  const int sls[4] = {8, 16, 32, 64};
  double best = 1e30;
  int best_bx = b->bx, best_sl = b->seglen;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  for (int bx : bxs) {
    if (!shape_supported(b->prec, bx)) continue;
    for (int sl : sls) {
      if (set_tiles(b, bx, sl)) continue;
      for (int k = 0; k < 2; ++k) {
        enqueue_batch_step(b, b->cur, b->stream);
        b->cur ^= 1;
      }
      cudaEventRecord(e0, b->stream);
      for (int k = 0; k < trial_steps; ++k) {
        enqueue_batch_step(b, b->cur, b->stream);
        b->cur ^= 1;
      }
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      const double us = 1e3 * ms / trial_steps;
      if (us < best) {
        best = us;
        best_bx = bx;
        best_sl = sl;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // restore
  for (size_t i = 0; i < b->ctx.size(); ++i)
    cudaMemcpyAsync(b->ctx[i]->f[cur0], saved[i], b->ctx[i]->state_bytes, cudaMemcpyDeviceToDevice, b->stream);
  cudaStreamSynchronize(b->stream);
  release();
  b->cur = cur0;
  for (mrtlb_ctx* c : b->ctx) c->cur = cur0;
  cudaMemsetAsync(b->err, 0, sizeof(int), b->stream);  // trial steps are not the user's
  b->graph_steps = graph_steps;
  int rc = set_tiles(b, best_bx, best_sl);
  if (rc) return rc;
  BCK(cudaGetLastError(), "tuning");
  if (cache_path && cache_path[0]) {
    if (FILE* fh = fopen(cache_path, "a")) {
      fprintf(fh, "%s %d %d %.3f\n", sig.c_str(), best_bx, best_sl, best);
      fclose(fh);
    }
  }
  if (bx_out) *bx_out = best_bx;
  if (seglen_out) *seglen_out = best_sl;
  return MRTLB_OK;
}

extern "C" const char* mrtlb_batch_last_error(const mrtlb_batch* b) {
  return b ? b->last_error.c_str() : "";
}

extern "C" void mrtlb_batch_destroy(mrtlb_batch* b) {
  if (!b) return;
  if (b->stream || b->cap) cudaStreamSynchronize(b->stream);
  drop_graphs(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->d_insts) cudaFree(b->d_insts);
  if (b->d_walls) cudaFree(b->d_walls);
  if (b->d_tiles) cudaFree(b->d_tiles);
  if (b->err) cudaFree(b->err);
  if (b->claim) cudaFree(b->claim);
  delete b;
}
