// ensemble.cu -- many independent lattices (D2Q9 and D3Q19 members of uneven sizes, fluxes,
// density ratios and thresholds) advanced by one persistent cooperative launch per call, captured
// in a CUDA graph, with the tiling picked by a measuring autotuner.
//
// Work list.  A step of a member is split into items: (member, tile, chunk of planes) exactly as
// the single-lattice step kernel splits it.  A D3Q19 item fills a 128-thread CTA (32 x 4 tile;
// four CTAs per SM, as the fastest single-lattice step); D2Q9 items are narrower and run G at a
// time in one CTA, one per group of 128/G threads (row tiles of 128/G cells), with their barrier
// rounds padded to the longest chunk of the pack.  Members store FP32 or FP64 populations, or
// all of them FP32 pairs with exact colour masses; a pack holds items of one storage only, so
// every barrier round of a CTA runs the same code.
// CTAs take items (or packs) from a counter, meet at a grid barrier after every step, and fold
// the per-item ledger partials of each member in item order (deterministic).  Every wait is
// bounded (4 s by default, settable from the host); a barrier that gives up sets the status
// word, the CTAs finish their loops and the host reports CGEVAP_ERR_TIMEOUT.  Paused members
// have no items: their state, site bytes and ledger stay as they are.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/cgevap.h"
#include "launch.h"
#include "sim.h"
#include "step_kernel.cuh"

using namespace cgevap;

namespace cgevap {

struct EnsMember {
  StepArgs a;           // geometry, physics and tiling of the member (pointers set per step)
  void* state[2];
  uint8_t* mask[2];
  DevLedger* ledger;
  int q;
  int storage;          // ST_F32 or ST_F64 (an all-F32X ensemble labels its members ST_F32)
  int item0, nitem;     // its items: [item0, item0 + nitem) of the concatenated list (0: paused)
};

struct EnsArgs {
  const EnsMember* members;
  int nmembers;
  const int4* items;     // (member, tile, chunk, planes) -- D3Q19 items first, then D2Q9 packs
  int n3;                // D3Q19 items
  int npack;             // D2Q9 packs of G items (missing ones have member -1)
  int nitems;            // all items (partials are indexed by item)
  double* part_removed;  // [2][nitems]
  long long* part_sites;  // [2][nitems]
  const int* cur;        // [nmembers] buffer holding each member's state at launch
  unsigned int* bar;     // [4]: arrivals, generation, work counters of even / odd steps
  int* status;
  int nsteps;
  unsigned long long barrier_ns;  // limit of one grid-barrier wait
  int skip_cta, skip_step;        // test hook: this CTA does not arrive after this step (-1: off)
};

// Grid-wide barrier of a cooperative launch; a wait gives up after limit_ns and sets *status.
// skip: this CTA does not arrive (test hook that makes the other CTAs' waits run out).
__device__ __forceinline__ void grid_barrier(unsigned int* bar, int* status,
                                             unsigned long long limit_ns, bool skip) {
  __syncthreads();
  if (threadIdx.x == 0 && !skip) {
    volatile unsigned int* vgen = bar + 1;
    const unsigned int gen = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(bar, 1u) + 1u;
    if (arrived == gridDim.x) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      unsigned long long t0, t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      while (*vgen == gen) {
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > limit_ns) {
          atomicExch(status, 1);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

constexpr int kEnsThreads = 128;  // threads per CTA
constexpr int kEnsTy = 4;         // D3Q19 item tile: 32 x kEnsTy columns

// Member storages a kernel instantiation handles: FP32 only, FP64 only, both, or FP32 pairs with
// exact colour masses only.
enum { kEnsF32 = 0, kEnsF64 = 1, kEnsMixed = 2, kEnsF32X = 3 };

// The FP32 storage code of the ensemble's FP32 members under MODE.
template <int MODE>
constexpr int ens_s32() {
  return MODE == kEnsF32X ? ST_F32X : ST_F32;
}

// Shared memory of one D2Q9 group / one D3Q19 item of storage S.
template <int G, int S>
constexpr int ens_group_smem() {
  return TileSmem<9, S, kEnsThreads / G, 1, 1>::BYTES;
}

template <int G, int MODE>
__global__ void __launch_bounds__(kEnsThreads, MODE == kEnsF32 || MODE == kEnsF32X ? 4 : 2)
    cg_ensemble_kernel(const __grid_constant__ EnsArgs E) {
  constexpr int NT = kEnsThreads;
  constexpr int S32 = ens_s32<MODE>();
  constexpr int GT = NT / G;  // threads per D2Q9 group
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ double gsum_d[NT / 32];
  __shared__ long long gsum_n[NT / 32];
  const int tid = threadIdx.x;
  const int grp = tid / GT, gtid = tid % GT;
  for (int step = 0; step < E.nsteps; ++step) {
    const int par = step & 1;
    double* pr = E.part_removed + (size_t)par * E.nitems;
    long long* ps = E.part_sites + (size_t)par * E.nitems;
    const int nwork = E.n3 + E.npack;
    // items are taken from a counter in list order (largest D3Q19 members first), so a CTA that
    // finishes early takes the next one: the step ends when the work does, not when the CTA with
    // the unluckiest static share does
    unsigned int* const next = E.bar + 2 + par;
    __shared__ int w_sh;
    for (;;) {
      if (tid == 0) w_sh = (int)atomicAdd(next, 1u);
      __syncthreads();
      const int w = w_sh;
      __syncthreads();  // every thread has read w before thread 0 takes the next one
      if (w >= nwork) break;
      long long n = 0;
      double d = 0.0;
      if (w < E.n3) {
        const int4 it = E.items[w];
        const EnsMember& M = E.members[it.x];
        StepArgs A = M.a;
        const int c = (E.cur[it.x] + step) & 1;
        A.pin = M.state[c];
        A.pout = M.state[c ^ 1];
        A.mask_in = M.mask[c];
        A.mask_out = M.mask[c ^ 1];
        const bool f64 = MODE == kEnsF64 || (MODE == kEnsMixed && M.storage == ST_F64);
        if (MODE != kEnsF64 && !f64)
          step_tile<19, S32, 32, kEnsTy, 1>(A, it.y, it.z, smem, n, d);
        else if (MODE == kEnsF64 || MODE == kEnsMixed)
          step_tile<19, ST_F64, 32, kEnsTy, 1>(A, it.y, it.z, smem, n, d);
        block_sum<NT>(n, d);
        if (tid == 0) {
          pr[w] = d;
          ps[w] = n;
        }
      } else {
        const int pack = w - E.n3;
        const int4 it = E.items[E.n3 + pack * G + grp];
        int iters = 0;
        for (int g = 0; g < G; ++g) iters = max(iters, E.items[E.n3 + pack * G + g].w);
        // the pack's storage: that of its first item, which is never a filler
        const bool f64 = MODE == kEnsF64 ||
                         (MODE == kEnsMixed && E.members[E.items[E.n3 + pack * G].x].storage == ST_F64);
        unsigned char* gs = smem + grp * (f64 ? ens_group_smem<G, ST_F64>() : ens_group_smem<G, S32>());
        if (it.x >= 0) {
          const EnsMember& M = E.members[it.x];
          StepArgs A = M.a;
          const int c = (E.cur[it.x] + step) & 1;
          A.pin = M.state[c];
          A.pout = M.state[c ^ 1];
          A.mask_in = M.mask[c];
          A.mask_out = M.mask[c ^ 1];
          if (MODE != kEnsF64 && !f64)
            step_tile<9, S32, GT, 1, 1>(A, it.y, it.z, gs, n, d, gtid, iters);
          else if (MODE == kEnsF64 || MODE == kEnsMixed)
            step_tile<9, ST_F64, GT, 1, 1>(A, it.y, it.z, gs, n, d, gtid, iters);
        } else {
          for (int r = 0; r < 1 + iters; ++r) __syncthreads();  // same barrier rounds, no work
        }
        // per-group sums: warp shuffles, then the group's warps in shared memory
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
          n += __shfl_down_sync(0xffffffffu, n, off);
          d += __shfl_down_sync(0xffffffffu, d, off);
        }
        if ((tid & 31) == 0) {
          gsum_d[tid >> 5] = d;
          gsum_n[tid >> 5] = n;
        }
        __syncthreads();
        if (gtid == 0 && it.x >= 0) {
          double s = 0.0;
          long long k = 0;
          for (int j = 0; j < GT / 32; ++j) {
            s += gsum_d[grp * (GT / 32) + j];
            k += gsum_n[grp * (GT / 32) + j];
          }
          pr[E.n3 + pack * G + grp] = s;
          ps[E.n3 + pack * G + grp] = k;
        }
        __syncthreads();
      }
    }
    grid_barrier(E.bar, E.status, E.barrier_ns,
                 (int)blockIdx.x == E.skip_cta && step == E.skip_step);
    // this step's counter is next used two steps on, after one more barrier
    if (blockIdx.x == 0 && tid == 0) E.bar[2 + par] = 0u;
    // a barrier that gave up ends the launch in every CTA (each waits at most once more)
    __shared__ int stop;
    if (tid == 0) stop = *(volatile int*)E.status;
    __syncthreads();
    if (stop) break;
    // fold this step's partials into each member's ledger (in item order)
    if (tid == 0) {
      for (int j = blockIdx.x; j < E.nmembers; j += gridDim.x) {
        const EnsMember& M = E.members[j];
        if (M.nitem == 0) continue;  // paused: its ledger does not move
        double s = 0.0;
        long long k = 0;
        for (int i = 0; i < M.nitem; ++i) {  // the member's items, through the index table
          const int idx = E.items[M.item0 + i].x;
          s += __ldcg(pr + idx);
          k += __ldcg(ps + idx);
        }
        DevLedger* led = M.ledger;
        led->evaporated += s;
        led->last_removed = s;
        led->site_steps += k;
        led->last_sites = k;
        led->steps += 1;
      }
    }
  }
}

// Dynamic shared memory of the ensemble kernel for group count G and member storages MODE.
template <int G, int MODE>
static int ens_smem() {
  constexpr int S32 = ens_s32<MODE>();
  constexpr int b32 = G * ens_group_smem<G, S32>() > TileSmem<19, S32, 32, kEnsTy, 1>::BYTES
                          ? G * ens_group_smem<G, S32>()
                          : TileSmem<19, S32, 32, kEnsTy, 1>::BYTES;
  constexpr int b64 = G * ens_group_smem<G, ST_F64>() > TileSmem<19, ST_F64, 32, kEnsTy, 1>::BYTES
                          ? G * ens_group_smem<G, ST_F64>()
                          : TileSmem<19, ST_F64, 32, kEnsTy, 1>::BYTES;
  return MODE == kEnsF32 || MODE == kEnsF32X ? b32 : (MODE == kEnsF64 ? b64 : (b32 > b64 ? b32 : b64));
}

template <int G, int MODE>
static const void* ens_fn() {
  return (const void*)cg_ensemble_kernel<G, MODE>;
}

}  // namespace cgevap

// ====================================================================== host side ===========

struct cgevap_ens {
  int n = 0;
  std::vector<cgevap_sim*> sims;
  std::vector<cgevap_params> params;
  std::vector<int> cur;  // host mirror of every member's current buffer
  cudaStream_t stream = nullptr;
  int device = 0;
  // device data
  EnsMember* d_members = nullptr;
  int4* d_items = nullptr;
  std::vector<EnsMember> h_members;  // host copy of the member table
  double* d_part_removed = nullptr;
  long long* d_part_sites = nullptr;
  int* d_cur = nullptr;
  unsigned int* d_bar = nullptr;
  int* d_status = nullptr;
  size_t items_cap = 0;
  int mode = kEnsF32;                  // member storages (kEnsF32 / kEnsF64 / kEnsMixed / kEnsF32X)
  std::vector<int> active;             // 0: member paused (no items)
  unsigned long long barrier_ns = 4000000000ull;
  int skip_cta = -1, skip_step = -1;   // test hook of the grid barrier
  // plan
  int groups = 4;        // D2Q9 items per CTA
  int pc3 = 16, pc2 = 32;
  int n3 = 0, npack = 0, nitems = 0;
  int grid = 0, smem = 0;
  // graph cache
  cudaGraphExec_t graph = nullptr;
  int graph_steps = -1;
  long long cells = 0;
  std::string err;
};



namespace {

int efail(cgevap_ens* e, int code, const std::string& m) {
  if (e) e->err = m;
  return code;
}

#define EN_CUDA(e, call)                                                                       \
  do {                                                                                         \
    cudaError_t r_ = (call);                                                                   \
    if (r_ != cudaSuccess)                                                                     \
      return efail((e), CGEVAP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(r_)); \
  } while (0)

const void* kernel_for_groups(int g, int mode) {
  switch (g * 4 + mode) {
    case 2 * 4 + kEnsF32: return ens_fn<2, kEnsF32>();
    case 4 * 4 + kEnsF32: return ens_fn<4, kEnsF32>();
    case 2 * 4 + kEnsF64: return ens_fn<2, kEnsF64>();
    case 4 * 4 + kEnsF64: return ens_fn<4, kEnsF64>();
    case 2 * 4 + kEnsMixed: return ens_fn<2, kEnsMixed>();
    case 4 * 4 + kEnsMixed: return ens_fn<4, kEnsMixed>();
    case 2 * 4 + kEnsF32X: return ens_fn<2, kEnsF32X>();
    case 4 * 4 + kEnsF32X: return ens_fn<4, kEnsF32X>();
    default: return nullptr;
  }
}
int smem_for_groups(int g, int mode) {
  switch (g * 4 + mode) {
    case 2 * 4 + kEnsF32: return ens_smem<2, kEnsF32>();
    case 4 * 4 + kEnsF32: return ens_smem<4, kEnsF32>();
    case 2 * 4 + kEnsF64: return ens_smem<2, kEnsF64>();
    case 4 * 4 + kEnsF64: return ens_smem<4, kEnsF64>();
    case 2 * 4 + kEnsMixed: return ens_smem<2, kEnsMixed>();
    case 4 * 4 + kEnsMixed: return ens_smem<4, kEnsMixed>();
    case 2 * 4 + kEnsF32X: return ens_smem<2, kEnsF32X>();
    case 4 * 4 + kEnsF32X: return ens_smem<4, kEnsF32X>();
    default: return 0;
  }
}

// The cached graph holds the launch's arguments: drop it when they change.
void drop_graph(cgevap_ens* e) {
  if (e->graph) {
    cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
    e->graph_steps = -1;
  }
}

// Build the item list and the member table for the current plan; (re)allocate partials.
int build_plan(cgevap_ens* e) {
  std::vector<EnsMember> mem(e->n);
  std::vector<int4> it3, it2;
  std::vector<std::vector<int4>> per2(e->n), per3(e->n);
  const int gt = kEnsThreads / e->groups;
  for (int j = 0; j < e->n; ++j) {
    SimView v;
    if (sim_view(e->sims[j], &v) != CGEVAP_OK) return efail(e, CGEVAP_ERR_ARG, "bad member");
    EnsMember& M = mem[j];
    std::memset(&M, 0, sizeof(M));
    M.q = e->params[j].q;
    M.storage = e->params[j].storage == CGEVAP_F64 ? ST_F64 : ST_F32;
    M.a.g = v.g;
    M.a.ph = v.ph;
    M.state[0] = v.state[0];
    M.state[1] = v.state[1];
    M.mask[0] = v.mask[0];
    M.mask[1] = v.mask[1];
    M.ledger = v.ledger;
    const int tx = M.q == 19 ? 32 : gt, ty = M.q == 19 ? kEnsTy : 1;
    const int pc = M.q == 19 ? e->pc3 : e->pc2;
    M.a.ntx = (v.g.na + tx - 1) / tx;
    M.a.nty = (v.g.nb + ty - 1) / ty;
    M.a.pc = std::min(pc, v.g.nm);
    const int nch = (v.g.nm + M.a.pc - 1) / M.a.pc;
    if (!e->active[j]) continue;  // paused: no items
    for (int t = 0; t < M.a.ntx * M.a.nty; ++t)
      for (int c = 0; c < nch; ++c) {
        const int planes = std::min(M.a.pc, v.g.nm - c * M.a.pc);
        (M.q == 19 ? per3[j] : per2[j]).push_back(make_int4(j, t, c, planes));
      }
  }
  // D3Q19 items largest-member first; D2Q9 items packed G at a time, by chunk length
  std::vector<int> order(e->n);
  for (int j = 0; j < e->n; ++j) order[j] = j;
  std::sort(order.begin(), order.end(), [&](int x, int y) {
    return mem[x].a.g.ncell > mem[y].a.g.ncell;
  });
  std::vector<int4> items;
  for (int j : order)
    for (const int4& v : per3[j]) items.push_back(v);
  const int n3 = (int)items.size();
  // D2Q9 items: FP32 members' packs, then FP64 members' packs (one storage per pack), each
  // padded with fillers (member -1) to whole packs
  std::vector<int4> flat2;
  for (int st : {ST_F32, ST_F64}) {
    std::vector<int4> part;
    for (int j : order)
      if (mem[j].storage == st)
        for (const int4& v : per2[j]) part.push_back(v);
    std::stable_sort(part.begin(), part.end(), [](const int4& x, const int4& y) { return x.w > y.w; });
    if (part.empty()) continue;
    while (part.size() % e->groups) part.push_back(make_int4(-1, 0, 0, 0));
    flat2.insert(flat2.end(), part.begin(), part.end());
  }
  for (const int4& v : flat2) items.push_back(v);
  // member -> its items (contiguous ranges are not guaranteed: record by scanning)
  // Partials are indexed by item; a member's fold walks a per-member index list stored after
  // the items (kept simple: re-order items so that each member's items are contiguous within
  // the D3Q19 part; D2Q9 members fold through the index table below).
  std::vector<int> fold_index;
  std::vector<int> first(e->n, 0), count(e->n, 0);
  for (int j = 0; j < e->n; ++j) {
    first[j] = (int)fold_index.size();
    for (int i = 0; i < (int)items.size(); ++i)
      if (items[i].x == j) fold_index.push_back(i);
    count[j] = (int)fold_index.size() - first[j];
  }
  e->n3 = n3;
  e->npack = (int)flat2.size() / e->groups;
  e->nitems = (int)items.size();
  // items buffer: the work items, then the fold index table (as int4.x)
  std::vector<int4> dev_items(items);
  for (int i : fold_index) dev_items.push_back(make_int4(i, 0, 0, 0));
  for (int j = 0; j < e->n; ++j) {
    mem[j].item0 = e->nitems + first[j];
    mem[j].nitem = count[j];
  }
  const size_t need = dev_items.size();
  if (need > e->items_cap) {
    cudaFree(e->d_items);
    cudaFree(e->d_part_removed);
    cudaFree(e->d_part_sites);
    e->d_items = nullptr;
    e->d_part_removed = nullptr;
    e->d_part_sites = nullptr;
    if (cudaMalloc(&e->d_items, need * sizeof(int4)) != cudaSuccess ||
        cudaMalloc(&e->d_part_removed, 2 * need * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&e->d_part_sites, 2 * need * sizeof(long long)) != cudaSuccess) {
      e->items_cap = 0;
      return efail(e, CGEVAP_ERR_OOM, "cannot allocate the ensemble work list");
    }
    e->items_cap = need;
  }
  EN_CUDA(e, cudaMemcpyAsync(e->d_items, dev_items.data(), need * sizeof(int4), cudaMemcpyHostToDevice, e->stream));
  e->h_members = mem;
  EN_CUDA(e, cudaMemcpyAsync(e->d_members, e->h_members.data(), e->n * sizeof(EnsMember),
                             cudaMemcpyHostToDevice, e->stream));
  // resident CTAs
  const void* fn = kernel_for_groups(e->groups, e->mode);
  e->smem = smem_for_groups(e->groups, e->mode);
  EN_CUDA(e, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, e->smem));
  int occ = 0, sms = 0;
  EN_CUDA(e, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kEnsThreads, e->smem));
  EN_CUDA(e, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, e->device));
  if (occ < 1) return efail(e, CGEVAP_ERR_UNSUPPORTED, "ensemble kernel does not fit on an SM");
  e->grid = std::min(occ * sms, std::max(1, e->n3 + e->npack));
  drop_graph(e);
  return CGEVAP_OK;
}

int launch(cgevap_ens* e, int nsteps) {
  EnsArgs a;
  std::memset(&a, 0, sizeof(a));
  a.members = e->d_members;
  a.nmembers = e->n;
  a.items = e->d_items;
  a.n3 = e->n3;
  a.npack = e->npack;
  a.nitems = e->nitems;
  a.part_removed = e->d_part_removed;
  a.part_sites = e->d_part_sites;
  a.cur = e->d_cur;
  a.bar = e->d_bar;
  a.status = e->d_status;
  a.nsteps = nsteps;
  a.barrier_ns = e->barrier_ns;
  a.skip_cta = e->skip_cta;
  a.skip_step = e->skip_step;
  cudaLaunchConfig_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = dim3(e->grid);
  cfg.blockDim = dim3(kEnsThreads);
  cfg.dynamicSmemBytes = e->smem;
  cfg.stream = e->stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  void* args[] = {&a};
  // arrivals, generation and work counters start at zero (a launch whose barrier gave up may
  // have left arrivals counted and counters set)
  EN_CUDA(e, cudaMemsetAsync(e->d_bar, 0, 4 * sizeof(unsigned int), e->stream));
  EN_CUDA(e, cudaLaunchKernelExC(&cfg, kernel_for_groups(e->groups, e->mode), args));
  return CGEVAP_OK;
}

void sync_member_cur(cgevap_ens* e, int nsteps) {
  for (int j = 0; j < e->n; ++j) {
    if (!e->active[j]) continue;
    e->cur[j] ^= (nsteps & 1);
    SimView v;
    sim_view(e->sims[j], &v);
    *v.cur = e->cur[j];
  }
}

}  // namespace

extern "C" {

int cgevap_ensemble_create(const cgevap_params* members, int n, cgevap_ens** out) {
  if (!out || !members || n < 1) return CGEVAP_ERR_ARG;
  *out = nullptr;
  cgevap_ens* e = new (std::nothrow) cgevap_ens();
  if (!e) return CGEVAP_ERR_OOM;
  e->n = n;
  cudaGetDevice(&e->device);
  int seen = 0;  // bit 0: an FP32 member, bit 1: an FP64 member, bit 2: an F32X member
  for (int j = 0; j < n; ++j) {
    const int st = members[j].storage;
    if (st != CGEVAP_F32 && st != CGEVAP_F64 && st != CGEVAP_F32X) {
      cgevap_ensemble_destroy(e);
      return CGEVAP_ERR_UNSUPPORTED;
    }
    seen |= st == CGEVAP_F64 ? 2 : (st == CGEVAP_F32X ? 4 : 1);
  }
  if ((seen & 4) && seen != 4) {  // F32X members only with one another
    cgevap_ensemble_destroy(e);
    return CGEVAP_ERR_UNSUPPORTED;
  }
  e->mode = seen == 4 ? kEnsF32X : (seen == 1 ? kEnsF32 : (seen == 2 ? kEnsF64 : kEnsMixed));
  e->active.assign(n, 1);
  for (int j = 0; j < n; ++j) {
    cgevap_sim* s = nullptr;
    int rc = cgevap_create(&members[j], &s);
    if (rc != CGEVAP_OK) {
      cgevap_ensemble_destroy(e);
      return rc;
    }
    e->sims.push_back(s);
    e->params.push_back(members[j]);
    e->cur.push_back(0);
  }
  if (cudaMalloc(&e->d_members, n * sizeof(EnsMember)) != cudaSuccess ||
      cudaMalloc(&e->d_cur, n * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&e->d_bar, 4 * sizeof(unsigned int)) != cudaSuccess ||
      cudaMalloc(&e->d_status, sizeof(int)) != cudaSuccess) {
    cgevap_ensemble_destroy(e);
    return CGEVAP_ERR_OOM;
  }
  cudaMemset(e->d_bar, 0, 4 * sizeof(unsigned int));
  cudaMemset(e->d_status, 0, sizeof(int));
  cudaMemset(e->d_cur, 0, n * sizeof(int));
  int rc = build_plan(e);
  if (rc == CGEVAP_OK && cudaStreamSynchronize(e->stream) != cudaSuccess) rc = CGEVAP_ERR_CUDA;
  if (rc != CGEVAP_OK) {
    cgevap_ensemble_destroy(e);
    return rc;
  }
  *out = e;
  return CGEVAP_OK;
}

int cgevap_ensemble_destroy(cgevap_ens* e) {
  if (!e) return CGEVAP_OK;
  cudaStreamSynchronize(e->stream);
  if (e->graph) cudaGraphExecDestroy(e->graph);
  for (cgevap_sim* s : e->sims) cgevap_destroy(s);
  void* ptrs[] = {e->d_members, e->d_items, e->d_part_removed, e->d_part_sites,
                  e->d_cur,     e->d_bar,   e->d_status};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete e;
  return CGEVAP_OK;
}

const char* cgevap_ensemble_last_error(const cgevap_ens* e) { return e ? e->err.c_str() : ""; }

int cgevap_ensemble_size(const cgevap_ens* e) { return e ? e->n : 0; }

long long cgevap_ensemble_cells(const cgevap_ens* e) {
  if (!e) return 0;
  long long c = 0;
  for (int j = 0; j < e->n; ++j)
    if (e->active[j]) c += (long long)e->params[j].nx * e->params[j].ny * e->params[j].nz;
  return c;
}

int cgevap_ensemble_set_active(cgevap_ens* e, int j, int active) {
  if (!e || j < 0 || j >= e->n || (active != 0 && active != 1)) return CGEVAP_ERR_ARG;
  if (e->active[j] == active) return CGEVAP_OK;
  int any = 0;
  for (int k = 0; k < e->n; ++k) any |= k == j ? active : e->active[k];
  if (!any) return efail(e, CGEVAP_ERR_ARG, "an ensemble needs at least one active member");
  EN_CUDA(e, cudaSetDevice(e->device));
  e->active[j] = active;
  return build_plan(e);
}

int cgevap_ensemble_set_barrier_timeout(cgevap_ens* e, int ms) {
  if (!e || ms < 1) return CGEVAP_ERR_ARG;
  e->barrier_ns = (unsigned long long)ms * 1000000ull;
  drop_graph(e);
  return CGEVAP_OK;
}

int cgevap_ensemble_debug_skip_arrival(cgevap_ens* e, int cta, int step) {
  if (!e || cta < -1 || (cta >= 0 && step < 0)) return CGEVAP_ERR_ARG;
  e->skip_cta = cta;
  e->skip_step = cta < 0 ? -1 : step;
  drop_graph(e);
  return CGEVAP_OK;
}

int cgevap_ensemble_grid(const cgevap_ens* e) { return e ? e->grid : 0; }

int cgevap_ensemble_member(cgevap_ens* e, int j, cgevap_sim** out) {
  if (!e || !out || j < 0 || j >= e->n) return CGEVAP_ERR_ARG;
  *out = e->sims[j];
  return CGEVAP_OK;
}

int cgevap_ensemble_set_stream(cgevap_ens* e, void* stream) {
  if (!e) return CGEVAP_ERR_ARG;
  e->stream = (cudaStream_t)stream;
  for (cgevap_sim* s : e->sims) cgevap_set_stream(s, stream);
  drop_graph(e);
  return CGEVAP_OK;
}

int cgevap_ensemble_step(cgevap_ens* e, int nsteps) {
  if (!e || nsteps < 0) return CGEVAP_ERR_ARG;
  if (nsteps == 0) return CGEVAP_OK;
  EN_CUDA(e, cudaSetDevice(e->device));
  for (cgevap_sim* s : e->sims)  // per-step work the persistent kernel does not do
    if (s->outlet_rho[0] > 0.0 || s->outlet_rho[1] > 0.0 || s->heat.on)
      return efail(e, CGEVAP_ERR_UNSUPPORTED, "ensemble members run neither outlets nor a heated flux");
  // the member table carries each member's flux, physics and solids of the moment, and the
  // buffer each state sits in; refresh both before the (graph) launch
  for (int j = 0; j < e->n; ++j) {
    SimView v;
    sim_view(e->sims[j], &v);
    e->h_members[j].a.ph = v.ph;
    e->h_members[j].a.g.links = v.g.links;
    e->cur[j] = *v.cur;
  }
  EN_CUDA(e, cudaMemcpyAsync(e->d_members, e->h_members.data(), e->n * sizeof(EnsMember),
                             cudaMemcpyHostToDevice, e->stream));
  EN_CUDA(e, cudaMemcpyAsync(e->d_cur, e->cur.data(), e->n * sizeof(int), cudaMemcpyHostToDevice,
                             e->stream));
  if (e->graph_steps != nsteps) {
    if (e->graph) cudaGraphExecDestroy(e->graph);
    e->graph = nullptr;
    cudaStream_t cap = nullptr;
    EN_CUDA(e, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaStream_t keep = e->stream;
    e->stream = cap;
    bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    int lrc = ok ? launch(e, nsteps) : CGEVAP_ERR_CUDA;
    ok = (cudaStreamEndCapture(cap, &g) == cudaSuccess) && ok && lrc == CGEVAP_OK;
    e->stream = keep;
    cudaStreamDestroy(cap);
    if (!ok || cudaGraphInstantiate(&e->graph, g, 0) != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      e->graph = nullptr;
      return efail(e, CGEVAP_ERR_CUDA, "cannot capture the ensemble launch in a graph");
    }
    cudaGraphDestroy(g);
    e->graph_steps = nsteps;
  }
  EN_CUDA(e, cudaGraphLaunch(e->graph, e->stream));
  sync_member_cur(e, nsteps);
  return CGEVAP_OK;
}

int cgevap_ensemble_status(cgevap_ens* e) {
  if (!e) return CGEVAP_ERR_ARG;
  int st = 0;
  EN_CUDA(e, cudaMemcpyAsync(&st, e->d_status, sizeof(int), cudaMemcpyDeviceToHost, e->stream));
  EN_CUDA(e, cudaStreamSynchronize(e->stream));
  if (st) {
    cudaMemsetAsync(e->d_status, 0, sizeof(int), e->stream);
    return efail(e, CGEVAP_ERR_TIMEOUT, "a grid barrier of the ensemble launch gave up");
  }
  return CGEVAP_OK;
}

int cgevap_ensemble_get_tuning(const cgevap_ens* e, int* groups, int* pc3d, int* pc2d) {
  if (!e) return CGEVAP_ERR_ARG;
  if (groups) *groups = e->groups;
  if (pc3d) *pc3d = e->pc3;
  if (pc2d) *pc2d = e->pc2;
  return CGEVAP_OK;
}

int cgevap_ensemble_set_tuning(cgevap_ens* e, int groups, int pc3d, int pc2d) {
  if (!e || (groups != 2 && groups != 4) || pc3d < 1 || pc2d < 1) return CGEVAP_ERR_ARG;
  e->groups = groups;
  e->pc3 = pc3d;
  e->pc2 = pc2d;
  return build_plan(e);
}

int cgevap_ensemble_autotune(cgevap_ens* e, int probe_steps, double* best_ms) {
  if (!e || probe_steps < 1) return CGEVAP_ERR_ARG;
  EN_CUDA(e, cudaSetDevice(e->device));
  // back up every member's state, site bytes and ledger; probes run on the real buffers
  std::vector<void*> bk_state(e->n), bk_mask(e->n), bk_led(e->n);
  std::vector<int> cur0(e->n);
  for (int j = 0; j < e->n; ++j) {
    SimView v;
    sim_view(e->sims[j], &v);
    cur0[j] = *v.cur;
    if (cudaMalloc(&bk_state[j], v.state_bytes) != cudaSuccess ||
        cudaMalloc(&bk_mask[j], v.ncell) != cudaSuccess ||
        cudaMalloc(&bk_led[j], sizeof(DevLedger)) != cudaSuccess) {
      for (int k = 0; k <= j; ++k) {
        cudaFree(bk_state[k]);
        cudaFree(bk_mask[k]);
        cudaFree(bk_led[k]);
      }
      return efail(e, CGEVAP_ERR_OOM, "no room to back up the members for autotuning");
    }
    cudaMemcpyAsync(bk_state[j], v.state[*v.cur], v.state_bytes, cudaMemcpyDeviceToDevice, e->stream);
    cudaMemcpyAsync(bk_mask[j], v.mask[*v.cur], v.ncell, cudaMemcpyDeviceToDevice, e->stream);
    cudaMemcpyAsync(bk_led[j], v.ledger, sizeof(DevLedger), cudaMemcpyDeviceToDevice, e->stream);
  }
  const int cand_g[] = {4, 2};
  const int cand_p3[] = {16, 32, 64, 128};
  // short D2Q9 chunks for few small members (more items to spread over the resident CTAs)
  const int cand_p2[] = {4, 8, 16, 32, 64};
  // a lattice kind with no active member leaves its chunk length (and, for D2Q9, the group
  // count) without effect: probe one value of it
  bool has3 = false, has2 = false;
  for (int j = 0; j < e->n; ++j)
    if (e->active[j]) (e->params[j].q == 19 ? has3 : has2) = true;
  double best = 1e300;
  int bg = e->groups, b3 = e->pc3, b2 = e->pc2;
  cudaEvent_t t0, t1;
  cudaEventCreate(&t0);
  cudaEventCreate(&t1);
  int rc = CGEVAP_OK;
  for (int g : cand_g)
    for (int p3 : cand_p3)
      for (int p2 : cand_p2) {
        if ((!has2 && (g != cand_g[0] || p2 != 16)) || (!has3 && p3 != cand_p3[0])) continue;
        e->groups = g;
        e->pc3 = p3;
        e->pc2 = p2;
        if ((rc = build_plan(e)) != CGEVAP_OK) goto done;
        if ((rc = cgevap_ensemble_step(e, 1)) != CGEVAP_OK) goto done;  // warm-up
        cudaEventRecord(t0, e->stream);
        if ((rc = cgevap_ensemble_step(e, probe_steps)) != CGEVAP_OK) goto done;
        cudaEventRecord(t1, e->stream);
        cudaEventSynchronize(t1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t0, t1);
        if (ms < best) {
          best = ms;
          bg = g;
          b3 = p3;
          b2 = p2;
        }
      }
done:
  cudaEventDestroy(t0);
  cudaEventDestroy(t1);
  // restore the members exactly as they were
  for (int j = 0; j < e->n; ++j) {
    SimView v;
    sim_view(e->sims[j], &v);
    *v.cur = cur0[j];
    e->cur[j] = cur0[j];
    cudaMemcpyAsync(v.state[cur0[j]], bk_state[j], v.state_bytes, cudaMemcpyDeviceToDevice, e->stream);
    cudaMemcpyAsync(v.mask[cur0[j]], bk_mask[j], v.ncell, cudaMemcpyDeviceToDevice, e->stream);
    cudaMemcpyAsync(v.ledger, bk_led[j], sizeof(DevLedger), cudaMemcpyDeviceToDevice, e->stream);
  }
  cudaStreamSynchronize(e->stream);
  for (int j = 0; j < e->n; ++j) {
    cudaFree(bk_state[j]);
    cudaFree(bk_mask[j]);
    cudaFree(bk_led[j]);
  }
  if (rc != CGEVAP_OK) return rc;
  e->groups = bg;
  e->pc3 = b3;
  e->pc2 = b2;
  if (best_ms) *best_ms = best / probe_steps;
  return build_plan(e);
}

}  // extern "C"
