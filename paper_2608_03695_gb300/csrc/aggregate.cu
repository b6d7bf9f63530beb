// Aggregation (Louvain/Leiden, Sec. 3.2): one node per refined
// sub-community, numbered by ascending sub-community label.  Contraction
// without a sort: the level's nodes are bucketed by new id (member lists),
// then one warp or block per new node walks its members' rows and sums the
// weights per neighbouring new node in a shared-memory table; rows with more
// than 4096 entries use tables in global scratch and are spread over the
// whole grid.  Self-loops are dropped: no key or check reads them, and Q is
// always evaluated on level 0.  The same pass sums the members' snapshot
// strengths k_{x,s}.  Rows are written once to an upper-bound layout and
// compacted.  The order of a row's entries is not defined; nothing that
// reads a level depends on it (sums are exact integers and every scan is
// order-free).  The initial label of a new node is the smallest new id
// inside its local-moving community.
#include <algorithm>
#include <cstring>

#include "../../include/mslice.h"
#include "solver.h"

namespace mslice {

namespace {

__global__ void k_present(const int32_t* sizeR, int32_t N, int32_t* flag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
    flag[i] = sizeR[i] > 0 ? 1 : 0;
}

constexpr int CW_BITS = 9;        // warp tier: rows with at most 256 entries / snapshot entries
constexpr int CW_WARPS = 8;
constexpr int CB_BITS = 13;       // block tier: at most 4096
constexpr int CB_THREADS = 256;
constexpr int CW_MAX = 1 << (CW_BITS - 1), CB_MAX = 1 << (CB_BITS - 1);

// Per node: its new id; per new node: members, stored entries and snapshot
// entries (upper bounds of its output).
__global__ void k_contract_prep(LevelDev g, const int32_t* R, const int32_t* newid, int32_t* xmap, int32_t* mcnt,
                                long long* dsum, int32_t* scnt) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = newid[R[v]];
    xmap[v] = x;
    atomicAdd(&mcnt[x], 1);
    atomicAdd((ull*)&dsum[x], (ull)(g.rowptr[v + 1] - g.rowptr[v]));
    int64_t b, e;
    slice_range(g, (int32_t)v, b, e);
    if (e > b) atomicAdd(&scnt[x], (int32_t)(e - b));
  }
}

__global__ void k_contract_members(int32_t N, const int32_t* xmap, const int64_t* moff, int32_t* mfill, int32_t* mem) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = xmap[v];
    mem[moff[x] + atomicAdd(&mfill[x], 1)] = (int32_t)v;
  }
}

// Slots of a big row's global table for n entries: every entry could be a
// distinct key, so twice n keeps the load at most one half (short probe
// sequences; the power of two above 2n used before took up to twice this).
__device__ __forceinline__ int64_t big_table_slots(int64_t n) { return 2 * n + 16; }

// Rows by size: tier 0 (<= CW_MAX), 1 (<= CB_MAX), 2 (larger; its tables of
// big_table_slots(size) slots in global scratch).
__global__ void k_contract_tier(int32_t Np, const long long* dsum, const int32_t* scnt, int32_t* lists,
                                int32_t* tcnt, int64_t* gsize, int64_t* ssize) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < Np; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t x = base + threadIdx.x;
    int t = -1;
    if (x < Np) {
      const long long need = max(dsum[x], (long long)scnt[x]);
      t = need <= CW_MAX ? 0 : (need <= CB_MAX ? 1 : 2);
      gsize[x] = t == 2 ? big_table_slots(dsum[x]) : 0;
      ssize[x] = t == 2 ? big_table_slots(scnt[x]) : 0;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, t);
    const int leader = __ffs(peers) - 1;
    int pos = 0;
    if (t >= 0 && lane == leader) pos = atomicAdd(&tcnt[t], __popc(peers));
    pos = __shfl_sync(peers, pos, leader);
    if (t >= 0) lists[(int64_t)t * Np + pos + __popc(peers & ((1u << lane) - 1u))] = (int32_t)x;
  }
}

// Insert-or-add into a table of `cap` (a power of two) slots.
__device__ __forceinline__ int64_t ctab_add(int32_t* hk, long long* hv, int64_t cap, int32_t key, long long w,
                                            bool& fresh) {
  const uint64_t mask = (uint64_t)cap - 1;
  const int bits = 63 - __clzll((long long)cap);
  uint64_t i = ((uint64_t)(uint32_t)key * 0x9E3779B97F4A7C15ull) >> (64 - bits);
  for (uint64_t p = 0; p <= mask; ++p) {
    const int32_t prev = atomicCAS(&hk[i], -1, key);
    if (prev == -1 || prev == key) {
      atomicAdd((ull*)&hv[i], (ull)w);
      fresh = prev == -1;
      return (int64_t)i;
    }
    i = (i + 1) & mask;
  }
  fresh = false;
  return -1;
}

// Insert-or-add into a global table of `cap` slots (any size): home by a
// multiplicative hash and a multiply-high range reduction, linear probing.
__device__ __forceinline__ int64_t gtab_add(int32_t* hk, long long* hv, int64_t cap, int32_t key, long long w,
                                            bool& fresh) {
  uint64_t i = __umul64hi((uint64_t)(uint32_t)key * 0x9E3779B97F4A7C15ull, (uint64_t)cap);
  for (int64_t p = 0; p < cap; ++p) {
    const int32_t prev = atomicCAS(&hk[i], -1, key);
    if (prev == -1 || prev == key) {
      atomicAdd((ull*)&hv[i], (ull)w);
      fresh = prev == -1;
      return (int64_t)i;
    }
    i = (i + 1 == (uint64_t)cap) ? 0 : i + 1;
  }
  fresh = false;
  return -1;
}

// One warp per new node x (tier 0).  Members are fetched 32 at a time with
// their row bounds; lanes stride over each member's entries.
__global__ void __launch_bounds__(CW_WARPS * 32)
    k_contract_warp(LevelDev g, const int32_t* xmap, const int64_t* moff, const int32_t* mem, const int32_t* list,
                    const int32_t* count_ptr, const int64_t* eoff, const int64_t* soff, int32_t* tcol, long long* tw,
                    int32_t* ecnt, int32_t* tsidx, long long* tsval, int32_t* scnt_out) {
  constexpr int SLOTS = 1 << CW_BITS;
  __shared__ int32_t hk[CW_WARPS][SLOTS];
  __shared__ long long hv[CW_WARPS][SLOTS];
  __shared__ uint16_t cl[CW_WARPS][SLOTS / 2];
  __shared__ int32_t ncl[CW_WARPS];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t* K = hk[w];
  long long* V = hv[w];
  uint16_t* CL = cl[w];
  for (int i = lane; i < SLOTS; i += 32) {
    K[i] = -1;
    V[i] = 0;
  }
  if (lane == 0) ncl[w] = 0;
  __syncwarp();
  const int count = *count_ptr;
  const int64_t warps = (int64_t)gridDim.x * CW_WARPS;
  for (int64_t idx = (int64_t)blockIdx.x * CW_WARPS + w; idx < count; idx += warps) {
    const int32_t x = list[idx];
    const int64_t mb = moff[x], me = moff[x + 1];
    int n = 0;
    for (int64_t j0 = mb; j0 < me; j0 += 32) {
      const int64_t jj = j0 + lane;
      int32_t mv = 0;
      int64_t rb = 0, re = 0;
      if (jj < me) {
        mv = mem[jj];
        rb = g.rowptr[mv];
        re = g.rowptr[mv + 1];
      }
      const int cm = (int)min((int64_t)32, me - j0);
      for (int t = 0; t < cm; ++t) {
        const int32_t v = __shfl_sync(0xffffffffu, mv, t);
        const int64_t b = __shfl_sync(0xffffffffu, rb, t), e = __shfl_sync(0xffffffffu, re, t);
        const Omega om = node_omega(g, v);
        for (int64_t base = b; base < e; base += 32) {
          const int64_t i = base + lane;
          bool fresh = false;
          int64_t slot = 0;
          if (i < e) {
            int32_t u;
            long long W;
            if (edge_at(g, i, u, W, om)) {
              const int32_t y = xmap[u];
              if (y != x) slot = ctab_add(K, V, SLOTS, y, W, fresh);
#if MSLICE_CHECKED
              if (y != x && slot < 0) atomicOr(g.chk, ERR_BOUNDS);
#endif
            }
          }
          const unsigned bal = __ballot_sync(0xffffffffu, fresh);
          if (fresh) CL[n + __popc(bal & ((1u << lane) - 1u))] = (uint16_t)slot;
          n += __popc(bal);
        }
      }
    }
    __syncwarp();
    const int64_t eo = eoff[x];
    for (int k = lane; k < n; k += 32) {
      const int slot = CL[k];
      tcol[eo + k] = K[slot];
      tw[eo + k] = V[slot];
      K[slot] = -1;
      V[slot] = 0;
    }
    if (lane == 0) ecnt[x] = n;
    __syncwarp();
    // snapshot strengths: lane per member
    for (int64_t j = mb + lane; j < me; j += 32) {
      const int32_t v = mem[j];
      int64_t b, e;
      slice_range(g, v, b, e);
      for (int64_t q = b; q < e; ++q) {
        int32_t sl;
        long long k;
        slice_entry(g, v, q, sl, k);
        bool fresh;
        const int64_t slot = ctab_add(K, V, SLOTS, sl, k, fresh);
#if MSLICE_CHECKED
            if (slot < 0) atomicOr(g.chk, ERR_BOUNDS);
#endif
        if (fresh) CL[atomicAdd(&ncl[w], 1)] = (uint16_t)slot;
      }
    }
    __syncwarp();
    const int ns = ncl[w];
    const int64_t so = soff[x];
    for (int k = lane; k < ns; k += 32) {
      const int slot = CL[k];
      tsidx[so + k] = K[slot];
      tsval[so + k] = V[slot];
      K[slot] = -1;
      V[slot] = 0;
    }
    __syncwarp();
    if (lane == 0) {
      scnt_out[x] = ns;
      ncl[w] = 0;
    }
    __syncwarp();
  }
}

// One block per new node x of tier 1: a table of 2^CB_BITS slots in shared
// memory.  Warps take members in turn; lanes stride over entries.  Blocks
// claim their rows one at a time from a counter (queue), which keeps them
// busy until the list is done whatever the spread of row sizes.
__global__ void __launch_bounds__(CB_THREADS)
    k_contract_block(LevelDev g, const int32_t* xmap, const int64_t* moff, const int32_t* mem, const int32_t* list,
                     const int32_t* count_ptr, const int64_t* eoff, const int64_t* soff, int32_t* tcol, long long* tw,
                     int32_t* ecnt, int32_t* tsidx, long long* tsval, int32_t* scnt_out, int32_t* queue) {
  extern __shared__ __align__(16) unsigned char csm[];
  __shared__ int32_t ncnt;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int NW = CB_THREADS / 32;
  const int count = *count_ptr;
  constexpr int64_t cap = (int64_t)1 << CB_BITS;
  long long* V = reinterpret_cast<long long*>(csm);
  int32_t* K = reinterpret_cast<int32_t*>(V + cap);
  uint32_t* CL = reinterpret_cast<uint32_t*>(K + cap);  // listed slots
  for (int64_t i = threadIdx.x; i < cap; i += blockDim.x) {
    K[i] = -1;
    V[i] = 0;
  }
  __shared__ int32_t claim;
  if (threadIdx.x == 0) claim = -1;
  for (int idx; (idx = block_claim(queue, count, &claim)) >= 0;) {
    const int32_t x = list[idx];
    if (threadIdx.x == 0) ncnt = 0;
    __syncthreads();
    const int64_t mb = moff[x], me = moff[x + 1];
    for (int64_t j = mb + w; j < me; j += NW) {
      const int32_t v = mem[j];
      const int64_t b = g.rowptr[v], e = g.rowptr[v + 1];
      const Omega om = node_omega(g, v);
      for (int64_t i = b + lane; i < e; i += 32) {
        int32_t u;
        long long W;
        if (edge_at(g, i, u, W, om)) {
          const int32_t y = xmap[u];
          if (y != x) {
            bool fresh;
            const int64_t slot = ctab_add(K, V, cap, y, W, fresh);
#if MSLICE_CHECKED
            if (slot < 0) atomicOr(g.chk, ERR_BOUNDS);
#endif
            if (fresh) CL[atomicAdd(&ncnt, 1)] = (uint32_t)slot;
          }
        }
      }
    }
    __syncthreads();
    const int n = ncnt;
    const int64_t eo = eoff[x];
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const uint32_t slot = CL[k];
      tcol[eo + k] = K[slot];
      tw[eo + k] = V[slot];
      K[slot] = -1;
      V[slot] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      ecnt[x] = n;
      ncnt = 0;
    }
    __syncthreads();
    for (int64_t j = mb + threadIdx.x; j < me; j += blockDim.x) {
      const int32_t v = mem[j];
      int64_t b, e;
      slice_range(g, v, b, e);
      for (int64_t q = b; q < e; ++q) {
        int32_t sl;
        long long k;
        slice_entry(g, v, q, sl, k);
        bool fresh;
        const int64_t slot = ctab_add(K, V, cap, sl, k, fresh);
#if MSLICE_CHECKED
            if (slot < 0) atomicOr(g.chk, ERR_BOUNDS);
#endif
        if (fresh) CL[atomicAdd(&ncnt, 1)] = (uint32_t)slot;
      }
    }
    __syncthreads();
    const int ns = ncnt;
    const int64_t so = soff[x];
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
      const uint32_t slot = CL[k];
      tsidx[so + k] = K[slot];
      tsval[so + k] = V[slot];
      K[slot] = -1;
      V[slot] = 0;
    }
    if (threadIdx.x == 0) scnt_out[x] = ns;
    __syncthreads();
  }
}

// Tier 2 (rows of more than CB_MAX entries) is spread over the whole grid:
// warps take the members of all such rows in turn and insert into the row's
// tables in global scratch (edges and snapshot strengths in separate tables,
// pre-filled with free slots), listing claimed slots with per-row counters;
// a second kernel writes each row out.  big: the tier's rows; mpre: prefix of
// their member counts (nbig + 1 entries).
__global__ void k_big_members(const int32_t* big, const int32_t* nbig_ptr, const int64_t* moff, int64_t* cnt) {
  const int nbig = *nbig_ptr;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nbig; i += (int64_t)gridDim.x * blockDim.x)
    cnt[i] = moff[big[i] + 1] - moff[big[i]];
}

// Members of tier-2 rows are taken BI_CHUNK at a time by a block, which sums
// their entries per target in shared memory first (the members of one coarse
// community mostly reach the same few others, so adding every entry straight
// into the global table serialised on a few slots) and then adds each
// distinct target once to the row's global table.  An entry whose probe in
// the shared table runs past BI_PROBES slots goes to the global table
// directly; sums are integers, so the split changes nothing.
constexpr int BI_BITS = 11, BI_SBITS = 8, BI_CHUNK = 64, BI_PROBES = 16;
constexpr size_t BI_SMEM = ((size_t)1 << BI_BITS) * (sizeof(int32_t) + sizeof(long long) + sizeof(uint16_t)) +
                           ((size_t)1 << BI_SBITS) * (sizeof(int32_t) + sizeof(long long) + sizeof(uint16_t));

// Insert-or-add into a shared table of 2^bits slots, listing a newly taken
// slot in L (n: its length); false when the probe limit is reached (nothing
// added).
__device__ __forceinline__ bool stab_add(int32_t* K, long long* V, uint16_t* L, int* n, int bits, int32_t key,
                                         long long w) {
  const unsigned mask = (1u << bits) - 1u;
  unsigned i = ((uint32_t)key * 0x9E3779B1u) >> (32 - bits);
  for (int p = 0; p < BI_PROBES; ++p) {
    const int32_t prev = atomicCAS(&K[i], -1, key);
    if (prev == -1 || prev == key) {
      atomicAdd((ull*)&V[i], (ull)w);
      if (prev == -1) L[atomicAdd(n, 1)] = (uint16_t)i;
      return true;
    }
    i = (i + 1) & mask;
  }
  return false;
}

__device__ __forceinline__ void big_add(int32_t* hk, long long* hv, uint32_t* hl, int64_t o, int64_t cap,
                                        int32_t* cnt, int32_t key, long long w, const LevelDev& g) {
  bool fresh;
  const int64_t slot = gtab_add(hk + o, hv + o, cap, key, w, fresh);
#if MSLICE_CHECKED
  if (slot < 0) atomicOr(g.chk, ERR_BOUNDS);
#endif
  if (fresh) hl[o + atomicAdd(cnt, 1)] = (uint32_t)slot;
}

__global__ void __launch_bounds__(256)
    k_big_insert(LevelDev g, const int32_t* xmap, const int64_t* moff, const int32_t* mem, const int32_t* big,
                 const int32_t* nbig_ptr, const int64_t* mpre, const int64_t* gofs, const int64_t* gsize, int32_t* gk,
                 long long* gv, uint32_t* gl, int32_t* gcnt, const int64_t* sofs, const int64_t* ssize, int32_t* sk,
                 long long* sv, uint32_t* sl, int32_t* scnt) {
  extern __shared__ __align__(16) unsigned char bi_smem[];
  constexpr int EB = 1 << BI_BITS, SB = 1 << BI_SBITS;
  long long* EV = reinterpret_cast<long long*>(bi_smem);
  long long* SV = EV + EB;
  int32_t* EK = reinterpret_cast<int32_t*>(SV + SB);
  int32_t* SK = EK + EB;
  uint16_t* EL = reinterpret_cast<uint16_t*>(SK + SB);
  uint16_t* SL = EL + EB;
  __shared__ int row_sh, ne, ns;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int i = threadIdx.x; i < EB; i += blockDim.x) {
    EK[i] = -1;
    EV[i] = 0;
  }
  for (int i = threadIdx.x; i < SB; i += blockDim.x) {
    SK[i] = -1;
    SV[i] = 0;
  }
  if (threadIdx.x == 0) ne = ns = 0;
  const int nbig = *nbig_ptr;
  const int64_t total = mpre[nbig];
  const int64_t chunks = (total + BI_CHUNK - 1) / BI_CHUNK;
  for (int64_t ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
    const int64_t f0 = ch * BI_CHUNK, f1 = f0 + BI_CHUNK < total ? f0 + BI_CHUNK : total;
    if (threadIdx.x == 0) {
      int lo = 0, hi = nbig - 1;  // the big row holding member f0
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (mpre[mid] <= f0) lo = mid; else hi = mid - 1;
      }
      row_sh = lo;
    }
    __syncthreads();
    // the rows overlapping [f0, f1), one at a time (block-uniform)
    for (int lo = row_sh; lo < nbig && mpre[lo] < f1; ++lo) {
      const int64_t a = mpre[lo] > f0 ? mpre[lo] : f0, b = mpre[lo + 1] < f1 ? mpre[lo + 1] : f1;
      const int32_t x = big[lo];
      const int64_t o = gofs[x], cap = gsize[x], so = sofs[x], scap = ssize[x];
      for (int64_t f = a + warp; f < b; f += nwarps) {
        const int32_t v = mem[moff[x] + (f - mpre[lo])];
        const Omega om = node_omega(g, v);
        for (int64_t i = g.rowptr[v] + lane; i < g.rowptr[v + 1]; i += 32) {
          int32_t u;
          long long W;
          if (edge_at(g, i, u, W, om)) {
            const int32_t y = xmap[u];
            if (y != x && !stab_add(EK, EV, EL, &ne, BI_BITS, y, W)) big_add(gk, gv, gl, o, cap, &gcnt[lo], y, W, g);
          }
        }
        int64_t sb, se;
        slice_range(g, v, sb, se);
        for (int64_t q = sb + lane; q < se; q += 32) {
          int32_t s;
          long long k;
          slice_entry(g, v, q, s, k);
          if (!stab_add(SK, SV, SL, &ns, BI_SBITS, s, k)) big_add(sk, sv, sl, so, scap, &scnt[lo], s, k, g);
        }
      }
      __syncthreads();
      const int me = ne, ms = ns;
      __syncthreads();  // every thread has the counts before they are reset
      if (threadIdx.x == 0) ne = ns = 0;
      for (int j = threadIdx.x; j < me; j += blockDim.x) {
        const int i = EL[j];
        big_add(gk, gv, gl, o, cap, &gcnt[lo], EK[i], EV[i], g);
        EK[i] = -1;
        EV[i] = 0;
      }
      for (int j = threadIdx.x; j < ms; j += blockDim.x) {
        const int i = SL[j];
        big_add(sk, sv, sl, so, scap, &scnt[lo], SK[i], SV[i], g);
        SK[i] = -1;
        SV[i] = 0;
      }
      __syncthreads();
    }
  }
}

__global__ void k_big_output(const int32_t* big, const int32_t* nbig_ptr, const int64_t* gofs, const int32_t* gk,
                             const long long* gv, const uint32_t* gl, const int32_t* gcnt, const int64_t* sofs,
                             const int32_t* sk,
                             const long long* sv, const uint32_t* sl, const int32_t* scnt, const int64_t* eoff,
                             const int64_t* soff, int32_t* tcol, long long* tw, int32_t* ecnt, int32_t* tsidx,
                             long long* tsval, int32_t* scnt_out) {
  const int nbig = *nbig_ptr;
  for (int i = blockIdx.x; i < nbig; i += gridDim.x) {
    const int32_t x = big[i];
    const int64_t o = gofs[x], eo = eoff[x], so = soff[x], sb = sofs[x];
    const int n = gcnt[i], ns = scnt[i];
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
      const uint32_t slot = gl[o + k];
      tcol[eo + k] = gk[o + slot];
      tw[eo + k] = gv[o + slot];
    }
    for (int k = threadIdx.x; k < ns; k += blockDim.x) {
      const uint32_t slot = sl[sb + k];
      tsidx[so + k] = sk[sb + slot];
      tsval[so + k] = sv[sb + slot];
    }
    if (threadIdx.x == 0) {
      ecnt[x] = n;
      scnt_out[x] = ns;
    }
  }
}

// Rows from the upper-bound layout to their final places (warp per row).
__global__ void k_contract_compact(int32_t Np, const int64_t* eoff, const int32_t* ecnt, const int64_t* rowptr,
                                   const int32_t* tcol, const long long* tw, int32_t* col, long long* W,
                                   const int64_t* soff, const int32_t* scnt, const int64_t* sptr,
                                   const int32_t* tsidx, const long long* tsval, int32_t* sidx, long long* sval) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t x = (((int64_t)blockIdx.x * blockDim.x) >> 5) + (threadIdx.x >> 5); x < Np; x += warps) {
    const int64_t a = eoff[x], o = rowptr[x];
    const int n = ecnt[x];
    for (int k = lane; k < n; k += 32) {
      col[o + k] = tcol[a + k];
      W[o + k] = tw[a + k];
    }
    const int64_t sa = soff[x], so = sptr[x];
    const int ns = scnt[x];
    for (int k = lane; k < ns; k += 32) {
      sidx[so + k] = tsidx[sa + k];
      sval[so + k] = tsval[sa + k];
    }
  }
}

__global__ void k_min_init(const int32_t* P, const int32_t* R, const int32_t* newid, int32_t N, int32_t* minid) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    atomicMin(&minid[P[v]], newid[R[v]]);
}

__global__ void k_next_labels(const int32_t* P, const int32_t* R, const int32_t* newid, const int32_t* minid,
                              int32_t N, int32_t* next) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    next[newid[R[v]]] = minid[P[v]];
}

// Batches: instance of every new node and the first new id of every instance.
__global__ void k_next_inst(LevelDev g, const int32_t* R, const int32_t* newid, int32_t* inst_next, int32_t* off_next) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < g.N; v += (int64_t)gridDim.x * blockDim.x) {
    const int32_t x = newid[R[v]];
    const int32_t i = g.inst[v];
    inst_next[x] = i;
    atomicMin(&off_next[i], x);
  }
}

__global__ void k_compose(const int32_t* R, const int32_t* newid, int64_t N0, int32_t* node_of0) {
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N0; v += (int64_t)gridDim.x * blockDim.x)
    node_of0[v] = newid[R[node_of0[v]]];
}

__global__ void k_max_deg(const int64_t* rowptr, int32_t N, int32_t* mx) {
  int32_t m = 0;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < N; v += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (int32_t)(rowptr[v + 1] - rowptr[v]));
  for (int o = 16; o; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(mx, m);
}

unsigned gsz(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

bool aggregate(Solver& S, const Level& L, const int32_t* P, Level& next, const std::string& slot,
               int32_t* next_labels, int32_t* node_of0, int64_t* checksum) {
  Ctx& c = *S.c;
  const int32_t N = L.d.N;
  // new ids = ranks of the present sub-community labels
  int32_t* flag = S.tmp32a;
  int32_t* newid = S.tmp32b;
  launch(c, k_present, dim3(gsz(N)), dim3(256), 0, (const int32_t*)S.sizeR, N, flag);
  int32_t* d_np = c.ws->get<int32_t>("ag_np", 1);
  scan_excl(c, flag, newid, N, d_np);
  const int32_t Np = *static_cast<const int32_t*>(readback(c, d_np, sizeof(int32_t)));
  if (Np == N) return false;

  // ---- contraction: member lists, rows summed per neighbouring new node ----
  const int64_t np1 = (int64_t)Np + 1;
  int32_t* xmap = c.ws->get<int32_t>("ag_xmap", N);
  int32_t* mcnt = c.ws->get<int32_t>("ag_mcnt", np1);
  int32_t* scnt = c.ws->get<int32_t>("ag_scnt", np1);
  long long* dsum = c.ws->get<long long>("ag_dsum", np1);
  check_cuda(cudaMemsetAsync(mcnt, 0, np1 * sizeof(int32_t), c.stream), "memset");
  check_cuda(cudaMemsetAsync(scnt, 0, np1 * sizeof(int32_t), c.stream), "memset");
  check_cuda(cudaMemsetAsync(dsum, 0, np1 * sizeof(long long), c.stream), "memset");
  launch(c, k_contract_prep, dim3(gsz(N)), dim3(256), 0, L.d, (const int32_t*)S.R, (const int32_t*)newid, xmap, mcnt,
         dsum, scnt);
  int64_t* moff = c.ws->get<int64_t>("ag_moff", np1);
  int64_t* eoff = c.ws->get<int64_t>("ag_eoff", np1);
  int64_t* soff = c.ws->get<int64_t>("ag_soff", np1);
  scan_excl(c, (const int32_t*)mcnt, moff, np1, (int64_t*)nullptr);
  scan_excl(c, (const int64_t*)dsum, eoff, np1, (int64_t*)nullptr);
  scan_excl(c, (const int32_t*)scnt, soff, np1, (int64_t*)nullptr);
  int32_t* mem = c.ws->get<int32_t>("ag_mem", N);
  check_cuda(cudaMemsetAsync(mcnt, 0, np1 * sizeof(int32_t), c.stream), "memset");
  launch(c, k_contract_members, dim3(gsz(N)), dim3(256), 0, N, (const int32_t*)xmap, (const int64_t*)moff, mcnt, mem);
  int32_t* lists = c.ws->get<int32_t>("ag_lists", 3 * (size_t)Np);
  int32_t* tcnt = c.ws->get<int32_t>("ag_tcnt", 4);
  int64_t* gsize = c.ws->get<int64_t>("ag_gsize", np1);
  int64_t* gofs = c.ws->get<int64_t>("ag_gofs", np1);
  int64_t* ssize = c.ws->get<int64_t>("ag_ssize", np1);
  int64_t* sofs = c.ws->get<int64_t>("ag_sofs", np1);
  check_cuda(cudaMemsetAsync(tcnt, 0, 4 * sizeof(int32_t), c.stream), "memset");
  check_cuda(cudaMemsetAsync(gsize + Np, 0, sizeof(int64_t), c.stream), "memset");
  check_cuda(cudaMemsetAsync(ssize + Np, 0, sizeof(int64_t), c.stream), "memset");
  launch(c, k_contract_tier, dim3(gsz(Np)), dim3(256), 0, Np, (const long long*)dsum, (const int32_t*)scnt, lists, tcnt,
         gsize, ssize);
  int64_t* d_gtot = c.ws->get<int64_t>("ag_gtot", 2);
  scan_excl(c, (const int64_t*)gsize, gofs, np1, d_gtot);
  scan_excl(c, (const int64_t*)ssize, sofs, np1, d_gtot + 1);
  struct {
    int32_t t[4];
    int64_t gtot, stot;
  } hd;
  check_cuda(cudaMemcpyAsync(c.pinned, tcnt, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream), "copy");
  check_cuda(cudaMemcpyAsync(static_cast<char*>(c.pinned) + 16, d_gtot, 2 * sizeof(int64_t), cudaMemcpyDeviceToHost,
                             c.stream), "copy");
  sync(c);
  std::memcpy(&hd, c.pinned, sizeof(hd));
  const int64_t cap = L.nnz > 0 ? L.nnz : 1;
  const int64_t scap = L.ns > 0 ? L.ns : 1;
  int32_t* tcol = c.ws->get<int32_t>("ag_tcol", cap);
  long long* tw = c.ws->get<long long>("ag_tw", cap);
  int32_t* tsidx = c.ws->get<int32_t>("ag_tsidx", scap);
  long long* tsval = c.ws->get<long long>("ag_tsval", scap);
  int32_t* ecnt = c.ws->get<int32_t>("ag_ecnt", np1);
  int32_t* scnt_out = c.ws->get<int32_t>("ag_scnt_out", np1);
  check_cuda(cudaMemsetAsync(ecnt + Np, 0, sizeof(int32_t), c.stream), "memset");
  check_cuda(cudaMemsetAsync(scnt_out + Np, 0, sizeof(int32_t), c.stream), "memset");
  if (hd.t[0] > 0)
    launch(c, k_contract_warp, dim3(152 * 4), dim3(CW_WARPS * 32), 0, L.d, (const int32_t*)xmap, (const int64_t*)moff,
           (const int32_t*)mem, (const int32_t*)lists, (const int32_t*)tcnt, (const int64_t*)eoff,
           (const int64_t*)soff, tcol, tw, ecnt, tsidx, tsval, scnt_out);
  const size_t cb_smem = ((size_t)1 << CB_BITS) * (sizeof(long long) + sizeof(int32_t)) +
                         (size_t)CB_MAX * sizeof(int32_t);
  if (hd.t[1] > 0) {
    check_cuda(cudaFuncSetAttribute(k_contract_block, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cb_smem),
               "attribute");
    int32_t* queue = c.ws->get<int32_t>("ag_queue", 1);
    check_cuda(cudaMemsetAsync(queue, 0, sizeof(int32_t), c.stream), "memset");
    launch(c, k_contract_block, dim3(152 * 2), dim3(CB_THREADS), cb_smem, L.d, (const int32_t*)xmap,
           (const int64_t*)moff, (const int32_t*)mem, (const int32_t*)(lists + Np), (const int32_t*)(tcnt + 1),
           (const int64_t*)eoff, (const int64_t*)soff, tcol, tw, ecnt, tsidx, tsval, scnt_out, queue);
  }
  if (hd.t[2] > 0) {
    if (hd.gtot > ((int64_t)1 << 31) * 8) fail(MSLICE_ENOMEM, "aggregation scratch too large");
    const int32_t nbig = hd.t[2];
    const int32_t* big = lists + 2 * (int64_t)Np;
    const int32_t* nbig_d = tcnt + 2;
    int32_t* gk = c.ws->get<int32_t>("ag_gk", hd.gtot);
    long long* gv = c.ws->get<long long>("ag_gv", hd.gtot);
    uint32_t* gl = c.ws->get<uint32_t>("ag_gl", hd.gtot);
    int32_t* sk = c.ws->get<int32_t>("ag_sk", hd.stot);
    long long* sv = c.ws->get<long long>("ag_sv", hd.stot);
    uint32_t* sl = c.ws->get<uint32_t>("ag_sl", hd.stot);
    int32_t* cnts = c.ws->get<int32_t>("ag_bigcnt", 2 * (size_t)nbig);
    int64_t* mcnt_big = c.ws->get<int64_t>("ag_bigm", (size_t)nbig + 1);
    int64_t* mpre = c.ws->get<int64_t>("ag_bigpre", (size_t)nbig + 1);
    check_cuda(cudaMemsetAsync(gk, 0xff, hd.gtot * sizeof(int32_t), c.stream), "memset");
    check_cuda(cudaMemsetAsync(gv, 0, hd.gtot * sizeof(long long), c.stream), "memset");
    check_cuda(cudaMemsetAsync(sk, 0xff, hd.stot * sizeof(int32_t), c.stream), "memset");
    check_cuda(cudaMemsetAsync(sv, 0, hd.stot * sizeof(long long), c.stream), "memset");
    check_cuda(cudaMemsetAsync(cnts, 0, 2 * (size_t)nbig * sizeof(int32_t), c.stream), "memset");
    check_cuda(cudaMemsetAsync(mcnt_big + nbig, 0, sizeof(int64_t), c.stream), "memset");
    launch(c, k_big_members, dim3(gsz(nbig)), dim3(256), 0, big, nbig_d, (const int64_t*)moff, mcnt_big);
    scan_excl(c, (const int64_t*)mcnt_big, mpre, (int64_t)nbig + 1, (int64_t*)nullptr);
    check_cuda(cudaFuncSetAttribute(k_big_insert, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BI_SMEM),
               "attribute");
    launch(c, k_big_insert, dim3(152 * 4), dim3(256), BI_SMEM, L.d, (const int32_t*)xmap, (const int64_t*)moff,
           (const int32_t*)mem, big, nbig_d, (const int64_t*)mpre, (const int64_t*)gofs, (const int64_t*)gsize, gk,
           gv, gl, cnts, (const int64_t*)sofs, (const int64_t*)ssize, sk, sv, sl, cnts + nbig);
    launch(c, k_big_output, dim3(std::min<int32_t>(nbig, 152 * 4)), dim3(256), 0, big, nbig_d,
           (const int64_t*)gofs, (const int32_t*)gk, (const long long*)gv, (const uint32_t*)gl,
           (const int32_t*)cnts, (const int64_t*)sofs, (const int32_t*)sk, (const long long*)sv, (const uint32_t*)sl,
           (const int32_t*)(cnts + nbig), (const int64_t*)eoff, (const int64_t*)soff, tcol, tw, ecnt, tsidx, tsval,
           scnt_out);
  }

  int64_t* rowptr = c.ws->get<int64_t>(slot + "_rowptr", (size_t)np1);
  int64_t* sptr = c.ws->get<int64_t>(slot + "_sptr", (size_t)np1);
  int64_t* d_tot = c.ws->get<int64_t>("ag_tot", 2);
  scan_excl(c, (const int32_t*)ecnt, rowptr, np1, d_tot);
  scan_excl(c, (const int32_t*)scnt_out, sptr, np1, d_tot + 1);
  const int64_t* tots = static_cast<const int64_t*>(readback(c, d_tot, 2 * sizeof(int64_t)));
  const int64_t mu = tots[0], ms = tots[1];
  int32_t* col = c.ws->get<int32_t>(slot + "_col", mu);
  long long* W = c.ws->get<long long>(slot + "_W", mu);
  int32_t* sidx = c.ws->get<int32_t>(slot + "_sidx", ms);
  long long* sval = c.ws->get<long long>(slot + "_sval", ms);
  launch(c, k_contract_compact, dim3(gsz((int64_t)Np * 32)), dim3(256), 0, Np, (const int64_t*)eoff,
         (const int32_t*)ecnt, (const int64_t*)rowptr, (const int32_t*)tcol, (const long long*)tw, col, W,
         (const int64_t*)soff, (const int32_t*)scnt_out, (const int64_t*)sptr, (const int32_t*)tsidx,
         (const long long*)tsval, sidx, sval);

  next.d = LevelDev{};
  next.d.N = Np;
  next.d.is0 = 0;
  next.d.on = L.d.on;
  next.d.od = L.d.od;
  next.d.global_null = L.d.global_null;
  next.d.on_i = L.d.on_i;
  next.d.od_i = L.d.od_i;
  next.d.chk = L.d.chk;
  if (L.d.inst) {
    int32_t* inst_next = c.ws->get<int32_t>(slot + "_inst", (size_t)Np);
    int32_t* off_next = c.ws->get<int32_t>(slot + "_ioff", (size_t)S.B + 1);
    fill_i32(c, off_next, Np, (int64_t)S.B + 1);
    launch(c, k_next_inst, dim3(gsz(N)), dim3(256), 0, L.d, (const int32_t*)S.R, (const int32_t*)newid, inst_next,
           off_next);
    next.d.inst = inst_next;
    next.d.inst_off = off_next;
  }
  next.d.rowptr = rowptr;
  next.d.col = col;
  next.d.W = W;
  next.nnz = mu;
  next.nnz_eff = mu;
  next.d.sptr = sptr;
  next.d.sidx = sidx;
  next.d.sval = sval;
  next.ns = ms;

  // ---- initial labels, level map ----
  int32_t* minid = flag;  // reuse
  fill_i32(c, minid, INT32_MAX, N);
  launch(c, k_min_init, dim3(gsz(N)), dim3(256), 0, P, (const int32_t*)S.R, (const int32_t*)newid, N, minid);
  launch(c, k_next_labels, dim3(gsz(N)), dim3(256), 0, P, (const int32_t*)S.R, (const int32_t*)newid,
         (const int32_t*)minid, N, next_labels);
  if (node_of0)
    launch(c, k_compose, dim3(gsz(S.N0)), dim3(256), 0, (const int32_t*)S.R, (const int32_t*)newid, S.N0, node_of0);
  int32_t* d_mx = c.ws->get<int32_t>("ag_mx", 1);
  check_cuda(cudaMemsetAsync(d_mx, 0, sizeof(int32_t), c.stream), "memset");
  launch(c, k_max_deg, dim3(gsz(Np)), dim3(256), 0, (const int64_t*)rowptr, Np, d_mx);
  next.max_deg = *static_cast<const int32_t*>(readback(c, d_mx, sizeof(int32_t)));
  if (checksum) *checksum = (int64_t)level_checksum(S, next);
  return true;
}

}  // namespace mslice
