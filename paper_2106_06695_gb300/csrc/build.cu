// Lattice construction on the GPU (Sec. 3.2 "Splat"; Eq. canon_simplex).
//
//  1. k_elevate      one thread per point: z = x / l, y = E z in H_d (triangular basis),
//                    nearest remainder-0 point, rank of residuals, sum fix, barycentric
//                    weights.  Every floating-point step is a single IEEE-rounded FP64
//                    operation (explicit _rn intrinsics, file built with -fmad=false) so
//                    the integer results are identical to any other correct FP64
//                    evaluation of the same expression order.
//  2. locality order points sorted by their enclosing remainder-0 cell (lexicographic
//                    over the leading coordinates, stable), so that neighbouring work
//                    touches neighbouring vertices.
//  3. k_insert       one thread per (point, vertex): lock-free open addressing in a
//                    power-of-two table of 64-bit slots (31-bit hash tag | owner entry);
//                    the full key of a slot is recomputed from its owner entry, and
//                    atomicMin keeps the earliest entry as owner.
//  4. numbering      vertex ids = first occurrence in locality order (owner flags +
//                    exclusive scan).
//  5. k_neighbours   per vertex and direction j: ids of v +- t u_j, u_j = (d+1) e_j - 1.
//  6. splat lists    (vertex, entry) pairs sorted stably by vertex id (radix sort) give
//                    each vertex the list of (point, weight) it gathers.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "sgp_internal.cuh"

namespace sgp {
namespace {

constexpr uint64_t kEmpty = ~0ull;

__device__ __forceinline__ uint64_t mix64(uint64_t h) {
  h ^= h >> 33;
  h *= 0xff51afd7ed558ccdull;
  h ^= h >> 33;
  h *= 0xc4ceb9fe1a85ec53ull;
  h ^= h >> 33;
  return h;
}
// Vertex-filter bit of a linear hash: its upper half (the linear hash's high bits mix every
// coordinate through the odd 64-bit multipliers), cheap for the filter test that every
// (vertex, direction) candidate makes; the table's slot and tag still come from mix64.
__device__ __forceinline__ uint32_t filter_hash(uint64_t h) { return (uint32_t)(h >> 32); }

uint64_t host_mix64(uint64_t h) {
  h ^= h >> 33;
  h *= 0xff51afd7ed558ccdull;
  h ^= h >> 33;
  h *= 0xc4ceb9fe1a85ec53ull;
  h ^= h >> 33;
  return h;
}
uint64_t host_coord_mult(int c) { return host_mix64(0x9e3779b97f4a7c15ull * (uint64_t)(c + 1)) | 1ull; }

// Vertex hash, linear in the integer key: lin(key) = sum_c A_c key_c (mod 2^64) with odd
// per-coordinate multipliers A_c, then mixed.  A lattice step u_j = (d+1) e_j - 1 moves
// lin by (d+1) A_j - sum_c A_c, so a neighbour's hash costs O(1) from the vertex's.
// The multipliers A_c = mix64(0x9e3779b97f4a7c15 (c + 1)) | 1, one table per device
// (constant memory: the lattice kernels read them with warp-uniform c).
__constant__ uint64_t c_coord_mult[kMaxD];
__device__ __forceinline__ uint64_t coord_mult(int c) { return c_coord_mult[c]; }

__device__ __forceinline__ uint64_t lin_hash(const int* key, int D) {
  uint64_t h = 0;
  for (int c = 0; c < D; ++c) h += coord_mult(c) * (uint64_t)(int64_t)key[c];
  return h;
}

// Coordinate c of vertex k of the simplex (rem0, rank): rem0 + k, minus d+1 where the
// coordinate's rank exceeds d - k (the canonical vertex s_k, coordinates permuted).
__device__ __forceinline__ int vertex_coord(const int16_t* rem0, const uint8_t* rank, int d,
                                            int k, int c) {
  return (int)rem0[c] + k - ((int)rank[c] > d - k ? d + 1 : 0);
}

// Does the vertex of entry `e` (locality-ordered point e / D, vertex e % D) equal key?
template <int MAXD>
__device__ __forceinline__ bool entry_has_key(uint32_t e, const int* key, int d,
                                              const int32_t* perm, const int16_t* rem0,
                                              const uint8_t* rank) {
  const int D = d + 1;
  const int64_t i = perm[e / D];
  const int k = (int)(e % D);
  const int16_t* r0 = rem0 + i * D;
  const uint8_t* rk = rank + i * D;
  for (int c = 0; c < D; ++c)
    if (vertex_coord(r0, rk, d, k, c) != key[c]) return false;
  return true;
}

// ---------------------------------------------------------------------------------
// 1. Elevation, enclosing simplex, barycentric weights.
// ---------------------------------------------------------------------------------
template <int MAXD>
__global__ void __launch_bounds__(128) k_elevate(const float* __restrict__ X,
                                                 const float* __restrict__ ls,
                                                 const double* __restrict__ f, int64_t n,
                                                 int d, int16_t* __restrict__ rem0_out,
                                                 uint8_t* __restrict__ rank_out,
                                                 float* __restrict__ w_out,
                                                 int* __restrict__ qmin, int* __restrict__ qmax,
                                                 unsigned* __restrict__ err, int inject_nan) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int D = d + 1;
  const double Dd = (double)D;
  double y[MAXD];
  int rem0[MAXD];
  int rank[MAXD];
  double b[MAXD + 1];
  bool bad = false;
  // y = E z, E's column j is (1, .., 1, -(j+1), 0, ..) / sqrt((j+1)(j+2)) times the scale;
  // f[j] already holds scale / sqrt((j+1)(j+2)).
  double sm = 0.0;
  for (int c = d; c >= 1; --c) {
    const float xv = X[i * d + (c - 1)];
    const float lv = ls[c - 1];
    if (!isfinite(xv) || !isfinite(lv) || !(lv > 0.f)) bad = true;
    const double z = __ddiv_rn((double)xv, (double)lv);
    const double cf = __dmul_rn(z, f[c - 1]);
    y[c] = __dsub_rn(sm, __dmul_rn((double)c, cf));
    sm = __dadd_rn(sm, cf);
  }
  y[0] = sm;
  if (inject_nan && i == 0) bad = true;  // SGP_FAULT=nan_input
  if (bad) {
    atomicOr(err, ERRBIT_NONFINITE);
    for (int c = 0; c < D; ++c) y[c] = 0.0;
  }
  // nearest remainder-0 point coordinate by coordinate (ties go down)
  int sum = 0;
  bool range = false;
  for (int c = 0; c < D; ++c) {
    const double q = __ddiv_rn(y[c], Dd);
    const double lo = floor(q);
    const double down = __dmul_rn(lo, Dd);
    const double up = __dadd_rn(down, Dd);
    const double r0 = (__dsub_rn(up, y[c]) < __dsub_rn(y[c], down)) ? up : down;
    if (!(fabs(r0) <= 32000.0)) {
      range = true;
      rem0[c] = 0;
    } else {
      rem0[c] = (int)r0;
    }
    sum += rem0[c];
  }
  if (range) {  // keep the rest of the computation in bounds; the build reports the error
    sum = 0;
    for (int c = 0; c < D; ++c) {
      y[c] = 0.0;
      rem0[c] = 0;
    }
  }
  // rank: strictly larger residuals, plus equal residuals at a lower index.  The residuals
  // are compared through an order-preserving integer image of their fp64 bits (-0 taken as
  // +0, no NaN here), the same order as the fp64 comparison at integer-compare cost.
  long long key[MAXD];
  for (int c = 0; c < D; ++c) {
    const long long bits = __double_as_longlong(__dadd_rn(__dsub_rn(y[c], (double)rem0[c]), 0.0));
    key[c] = bits ^ ((bits >> 63) & 0x7fffffffffffffffLL);
  }
  for (int c = 0; c < D; ++c) {
    const long long kc = key[c];
    int rk = 0;
    for (int c2 = 0; c2 < c; ++c2) rk += key[c2] >= kc ? 1 : 0;
    for (int c2 = c + 1; c2 < D; ++c2) rk += key[c2] > kc ? 1 : 0;
    rank[c] = rk;
  }
  // move rem0 onto H_d (coordinate sum 0)
  const int h = sum / D;
  for (int c = 0; c < D; ++c) {
    rank[c] += h;
    if (rank[c] < 0) {
      rank[c] += D;
      rem0[c] += D;
    } else if (rank[c] > d) {
      rank[c] -= D;
      rem0[c] -= D;
    }
    rank[c] = min(max(rank[c], 0), d);  // already true when sum(y) = 0; guards the indexing
  }
  for (int c = 0; c <= D; ++c) b[c] = 0.0;
  for (int c = 0; c < D; ++c) {
    const double v = __ddiv_rn(__dsub_rn(y[c], (double)rem0[c]), Dd);
    b[d - rank[c]] = __dadd_rn(b[d - rank[c]], v);
    b[D - rank[c]] = __dsub_rn(b[D - rank[c]], v);
  }
  b[0] = __dadd_rn(b[0], __dadd_rn(1.0, b[D]));
  if (range) atomicOr(err, ERRBIT_RANGE);
  for (int c = 0; c < D; ++c) {
    rem0_out[i * D + c] = (int16_t)rem0[c];
    rank_out[i * D + c] = (uint8_t)rank[c];
    w_out[i * D + c] = __double2float_rn(b[c]);
  }
  const unsigned active = __activemask();
  const int lane = threadIdx.x & 31;
  const bool leader = lane == __ffs(active) - 1;
  for (int c = 0; c < d; ++c) {
    const int q = rem0[c] / D;  // rem0 is a multiple of D: exact
    const int qlo = __reduce_min_sync(active, q);
    const int qhi = __reduce_max_sync(active, q);
    if (leader) {
      atomicMin(&qmin[c], qlo);
      atomicMax(&qmax[c], qhi);
    }
  }
}

// ---------------------------------------------------------------------------------
// 2. Locality key: the remainder-0 cell's leading coordinates packed MSB-first.
// ---------------------------------------------------------------------------------
struct CellPack {
  int ncoord;
  int shift[kMaxD];
  int qmin[kMaxD];
};

__global__ void k_point_key(const int16_t* __restrict__ rem0, int64_t n, int D, CellPack pk,
                            uint32_t* __restrict__ key, uint32_t* __restrict__ val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t k = 0;
  for (int c = 0; c < pk.ncoord; ++c)
    k |= (uint32_t)((int)rem0[i * D + c] / D - pk.qmin[c]) << pk.shift[c];
  key[i] = k;
  val[i] = (uint32_t)i;
}

// ---------------------------------------------------------------------------------
// 3. Hash insert.
// ---------------------------------------------------------------------------------
template <int MAXD>
__global__ void __launch_bounds__(256) k_insert(const int32_t* __restrict__ perm,
                                                const int16_t* __restrict__ rem0,
                                                const uint8_t* __restrict__ rank, int64_t nD,
                                                int d, unsigned long long* __restrict__ table,
                                                uint64_t mask, int32_t* __restrict__ entry_slot,
                                                unsigned* __restrict__ err) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nD) return;
  const int D = d + 1;
  const int64_t i = perm[e / D];
  const int k = (int)(e % D);
  int key[MAXD];
  for (int c = 0; c < D; ++c) key[c] = vertex_coord(rem0 + i * D, rank + i * D, d, k, c);
  const uint64_t h = mix64(lin_hash(key, D));
  const uint32_t tag = (uint32_t)(h >> 33);
  const unsigned long long mine = ((unsigned long long)tag << 32) | (uint32_t)e;
  uint64_t slot = h & mask;
  for (uint64_t probe = 0; probe <= mask; ++probe) {
    const unsigned long long prev = atomicCAS(&table[slot], kEmpty, mine);
    if (prev == kEmpty) {
      entry_slot[e] = (int32_t)slot;
      return;
    }
    if ((uint32_t)(prev >> 32) == tag &&
        entry_has_key<MAXD>((uint32_t)prev, key, d, perm, rem0, rank)) {
      atomicMin(&table[slot], mine);
      entry_slot[e] = (int32_t)slot;
      return;
    }
    slot = (slot + 1) & mask;
  }
  atomicOr(err, ERRBIT_HASH_FULL);
  entry_slot[e] = -1;
}

// ---------------------------------------------------------------------------------
// 4. Numbering: owner flags, then ids by scan, then slot -> id and vertex keys.
// ---------------------------------------------------------------------------------
__global__ void k_owner_flags(const int32_t* __restrict__ entry_slot,
                              const unsigned long long* __restrict__ table, int64_t nD,
                              uint32_t* __restrict__ flags) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nD) return;
  const int32_t s = entry_slot[e];
  flags[e] = (s >= 0 && (uint32_t)table[s] == (uint32_t)e) ? 1u : 0u;
}

__global__ void k_assign_ids(const uint32_t* __restrict__ scanned,
                             const int32_t* __restrict__ entry_slot,
                             const unsigned long long* __restrict__ table,
                             const int32_t* __restrict__ perm, const int16_t* __restrict__ rem0,
                             const uint8_t* __restrict__ rank, int64_t nD, int d,
                             int32_t* __restrict__ slot_id, int16_t* __restrict__ keys,
                             uint64_t* __restrict__ vhash, int2* __restrict__ vrange,
                             uint32_t* __restrict__ bloom, uint64_t bloom_mask) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nD) return;
  const int32_t s = entry_slot[e];
  if (s < 0 || (uint32_t)table[s] != (uint32_t)e) return;
  const int D = d + 1;
  const uint32_t id = scanned[e];
  slot_id[s] = (int32_t)id;
  const int64_t i = perm[e / D];
  const int k = (int)(e % D);
  uint64_t h = 0;
  int lo = 1 << 30, hi = -(1 << 30);
  int16_t* row = keys + (int64_t)id * D;
  // the row's coordinates, stored two per 4-byte word where the row is 4-byte aligned
  int c = 0;
  if ((reinterpret_cast<uintptr_t>(row) & 3u) != 0) {
    const int x = vertex_coord(rem0 + i * D, rank + i * D, d, k, 0);
    row[0] = (int16_t)x;
    h += coord_mult(0) * (uint64_t)(int64_t)x;
    lo = min(lo, x);
    hi = max(hi, x);
    c = 1;
  }
  for (; c + 1 < D; c += 2) {
    const int x0 = vertex_coord(rem0 + i * D, rank + i * D, d, k, c);
    const int x1 = vertex_coord(rem0 + i * D, rank + i * D, d, k, c + 1);
    *reinterpret_cast<uint32_t*>(row + c) =
        (uint32_t)(uint16_t)(int16_t)x0 | ((uint32_t)(uint16_t)(int16_t)x1 << 16);
    h += coord_mult(c) * (uint64_t)(int64_t)x0 + coord_mult(c + 1) * (uint64_t)(int64_t)x1;
    lo = min(lo, min(x0, x1));
    hi = max(hi, max(x0, x1));
  }
  if (c < D) {
    const int x = vertex_coord(rem0 + i * D, rank + i * D, d, k, c);
    row[c] = (int16_t)x;
    h += coord_mult(c) * (uint64_t)(int64_t)x;
    lo = min(lo, x);
    hi = max(hi, x);
  }
  vhash[id] = h;
  vrange[id] = make_int2(lo, hi);
  const uint64_t b = filter_hash(h) & bloom_mask;  // the vertex's filter bit
  atomicOr(&bloom[b >> 5], 1u << (b & 31));
}

__global__ void k_entry_ids(const int32_t* __restrict__ entry_slot,
                            const int32_t* __restrict__ slot_id,
                            const int32_t* __restrict__ perm, const float* __restrict__ w_user,
                            const uint8_t* __restrict__ rank_user, int64_t nD, int D,
                            int32_t* __restrict__ idx, float* __restrict__ w,
                            uint8_t* __restrict__ rank) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nD) return;
  const int32_t s = entry_slot[e];
  idx[e] = s >= 0 ? slot_id[s] : 0;
  const int64_t u = (int64_t)perm[e / D] * D + (e % D);
  w[e] = w_user[u];
  rank[e] = rank_user[u];
}

// ---------------------------------------------------------------------------------
// 5. Neighbour table.
// ---------------------------------------------------------------------------------
// Does the vertex of entry `e` equal keys[v] + step u_j?  (the owner entry's key is
// recomputed from its point's rem0 and rank)
__device__ __forceinline__ bool entry_is_neighbour(uint32_t e, const int16_t* __restrict__ kv,
                                                   int j, int step, int d,
                                                   const int32_t* __restrict__ perm,
                                                   const int16_t* __restrict__ rem0,
                                                   const uint8_t* __restrict__ rank) {
  const int D = d + 1;
  const int64_t i = perm[e / D];
  const int k = (int)(e % D);
  for (int c = 0; c < D; ++c) {
    const int want = (int)kv[c] + step * ((c == j ? D : 0) - 1);
    if (vertex_coord(rem0 + i * D, rank + i * D, d, k, c) != want) return false;
  }
  return true;
}

// One thread per vertex, all directions j: ids of v -+ t u_j, t = 1..r, and hasnb[j / 32]
// [v] bit j % 32: whether v has a neighbour along j.  The neighbour's
// hash comes from the vertex's linear hash in O(1) (sum_A = sum_c A_c); most absent
// neighbours stop at the vertex filter (one bit per hash, sized to stay in L2); the key
// itself is read only to confirm a tag match.  The filter words of kNbrGroup directions
// (both signs) are loaded together before any of them is tested, so that their latencies
// overlap.  A neighbour outside the int16 key range does not exist.  counts[j]
// accumulates the vertices with a neighbour along j.
constexpr int kNbrGroup = 8;
__global__ void __launch_bounds__(256) k_neighbours(
    const int16_t* __restrict__ keys, const uint64_t* __restrict__ vhash,
    const int2* __restrict__ vrange, int64_t m, int d, int r, uint64_t sum_A,
    const unsigned long long* __restrict__ table, uint64_t mask,
    const int32_t* __restrict__ slot_id, const int32_t* __restrict__ perm,
    const int16_t* __restrict__ rem0, const uint8_t* __restrict__ rank,
    const uint32_t* __restrict__ bloom, uint64_t bloom_mask, int32_t* __restrict__ nbr,
    unsigned long long* __restrict__ counts, uint32_t* __restrict__ hasnb) {
  __shared__ unsigned block_count[kMaxD];  // this block's vertices with a neighbour along j
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int D = d + 1;
  for (int j = threadIdx.x; j < D; j += blockDim.x) block_count[j] = 0;
  __syncthreads();
  const bool live = v < m;
  const uint64_t hv = live ? vhash[v] : 0;
  const int2 rg = live ? vrange[v] : make_int2(0, 0);
  const int16_t* kv = keys + (live ? v : 0) * D;
  uint32_t word = 0;  // bits j % 32 of the directions with a neighbour, 32 at a time
  for (int j0 = 0; j0 < D; j0 += kNbrGroup) {
    uint32_t any = 0;  // bit q: a neighbour along j0 + q
    for (int t = 1; t <= r; ++t) {
      // filter bits of the group's 2 kNbrGroup candidates: bit 2 q + sg
      uint32_t hits = 0;
#pragma unroll
      for (int q = 0; q < kNbrGroup; ++q) {
        const int j = j0 + q;
        // t lin(u_j): the hash moves by -t lin(u_j) (sg = 0) or + t lin(u_j) (sg = 1)
        const uint64_t tdj = (uint64_t)t * ((uint64_t)D * coord_mult(j < D ? j : 0) - sum_A);
#pragma unroll
        for (int sg = 0; sg < 2; ++sg) {
          const uint64_t b = filter_hash(sg ? hv + tdj : hv - tdj) & bloom_mask;
          const uint32_t word = (live && j < D) ? __ldg(bloom + (b >> 5)) : 0u;
          hits |= ((word >> (b & 31)) & 1u) << (2 * q + sg);
        }
      }
      // absent unless a filter hit is confirmed in the table (streaming stores: the table
      // is written once, and the vertex filter should keep its place in L2)
      if (live) {
        const int64_t sj = (int64_t)2 * r * m;  // from direction j to j + 1
        int32_t* p0 = nbr + ((int64_t)j0 * 2 * r + 2 * (t - 1)) * m + v;
#pragma unroll
        for (int q = 0; q < kNbrGroup; ++q)
          if (j0 + q < D) {
            __stcs(p0 + q * sj, -1);
            __stcs(p0 + q * sj + m, -1);
          }
      }
      while (hits) {
        const int bit = __ffs(hits) - 1;
        hits &= hits - 1;
        const int q = bit >> 1, sg = bit & 1, j = j0 + q;
        const int step = sg ? t : -t;
        // every coordinate moves by -step except j, which moves by d step
        bool in_range = rg.x - t * d >= -32768 && rg.y + t * d <= 32767;
        if (!in_range) {
          in_range = true;
          for (int c = 0; c < D; ++c) {
            const int x = (int)kv[c] + step * ((c == j ? D : 0) - 1);
            in_range = in_range && x >= -32768 && x <= 32767;
          }
        }
        if (!in_range) continue;
        const uint64_t tdj = (uint64_t)t * ((uint64_t)D * coord_mult(j) - sum_A);
        const uint64_t h = mix64(sg ? hv + tdj : hv - tdj);
        const uint32_t tag = (uint32_t)(h >> 33);
        uint64_t slot = h & mask;
        for (uint64_t probe = 0; probe <= mask; ++probe) {
          const unsigned long long cur = table[slot];
          if (cur == kEmpty) break;
          if ((uint32_t)(cur >> 32) == tag &&
              entry_is_neighbour((uint32_t)cur, kv, j, step, d, perm, rem0, rank)) {
            nbr[(((int64_t)j * r + (t - 1)) * 2 + sg) * m + v] = slot_id[slot];
            any |= 1u << q;
            break;
          }
          slot = (slot + 1) & mask;
        }
      }
    }
    // vertices with a neighbour along j: one shared-memory add per warp, one global add
    // per block at the end
#pragma unroll
    for (int q = 0; q < kNbrGroup; ++q) {
      if (j0 + q >= D) break;
      const unsigned with = __ballot_sync(0xffffffffu, (any >> q) & 1u);
      if (with && (int)(threadIdx.x & 31) == __ffs(with) - 1)
        atomicAdd(&block_count[j0 + q], (unsigned)__popc(with));
    }
    word |= any << (j0 & 31);
    if (((j0 + kNbrGroup) & 31) == 0 || j0 + kNbrGroup >= D) {
      if (live) hasnb[(int64_t)(j0 >> 5) * m + v] = word;
      word = 0;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < D; j += blockDim.x)
    if (block_count[j]) atomicAdd(&counts[j], (unsigned long long)block_count[j]);
}

// Direction lists: thread per vertex, reading its direction bits (32 directions per word).
// A block first counts, per warp and direction, its vertices with a neighbour along the
// direction, takes one slot range per direction with one atomic, then each warp writes its
// vertices at its prefix within that range.  The order of a list is immaterial to the
// blur, which updates its vertices independently.
constexpr int kFillThreads = 512;
__global__ void __launch_bounds__(kFillThreads) k_active_fill(
    const uint32_t* __restrict__ hasnb, int64_t m, int D, const int64_t* __restrict__ off,
    unsigned long long* __restrict__ fill, int32_t* __restrict__ act) {
  constexpr int kWarps = kFillThreads / 32;
  __shared__ unsigned wpos[kWarps][kMaxD];  // counts, then each warp's offset in the list
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = v < m;
  const int lane = (int)(threadIdx.x & 31), warp = (int)(threadIdx.x >> 5);
  for (int e = threadIdx.x; e < kWarps * kMaxD; e += blockDim.x) (&wpos[0][0])[e] = 0;
  __syncthreads();
  for (int w = 0; w * 32 < D; ++w) {
    const uint32_t bits = live ? hasnb[(int64_t)w * m + v] : 0u;
    uint32_t seen = __reduce_or_sync(0xffffffffu, bits);
    while (seen) {
      const int b = __ffs(seen) - 1;
      seen &= seen - 1;
      const unsigned with = __ballot_sync(0xffffffffu, (bits >> b) & 1u);
      if (lane == 0) wpos[warp][w * 32 + b] = (unsigned)__popc(with);
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < D; j += blockDim.x) {
    unsigned total = 0;
    for (int q = 0; q < kWarps; ++q) total += wpos[q][j];
    if (total == 0) continue;
    unsigned run = (unsigned)atomicAdd(&fill[j], (unsigned long long)total);
    for (int q = 0; q < kWarps; ++q) {
      const unsigned c = wpos[q][j];
      wpos[q][j] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int w = 0; w * 32 < D; ++w) {
    const uint32_t bits = live ? hasnb[(int64_t)w * m + v] : 0u;
    uint32_t seen = __reduce_or_sync(0xffffffffu, bits);
    while (seen) {
      const int b = __ffs(seen) - 1;
      seen &= seen - 1;
      const int j = w * 32 + b;
      const bool on = (bits >> b) & 1u;
      const unsigned with = __ballot_sync(0xffffffffu, on);
      if (on) act[off[j] + wpos[warp][j] + __popc(with & ((1u << lane) - 1u))] = (int32_t)v;
    }
  }
}

// ---------------------------------------------------------------------------------
// 6. Splat lists.
// ---------------------------------------------------------------------------------
__global__ void k_splat_items(const uint32_t* __restrict__ sorted_entries,
                              const float* __restrict__ w,
                              int64_t nD, int D, int2* __restrict__ items) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nD) return;
  const uint32_t e = sorted_entries[p];
  items[p] = make_int2((int)(e / D), __float_as_int(w[e]));
}

// Segment counts per vertex: total segments, partial slots, medium / huge flags.
__global__ void k_seg_count(const int32_t* __restrict__ row_ptr, int64_t m,
                            uint32_t* __restrict__ nseg, uint32_t* __restrict__ nslot,
                            uint32_t* __restrict__ med, uint32_t* __restrict__ huge) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= m) return;
  const int len = row_ptr[v + 1] - row_ptr[v];
  const uint32_t c = (uint32_t)((len + kSplatSeg - 1) / kSplatSeg);
  nseg[v] = c;
  nslot[v] = c > 1 ? c : 0u;
  med[v] = (c > 1 && c <= (uint32_t)kSplatMedSegs) ? 1u : 0u;
  huge[v] = c > (uint32_t)kSplatMedSegs ? 1u : 0u;
}

// After the exclusive scans: write every segment and the fix-up row lists.
__global__ void k_seg_fill(const int32_t* __restrict__ row_ptr, int64_t m,
                           const uint32_t* __restrict__ seg_off,
                           const uint32_t* __restrict__ slot_off,
                           const uint32_t* __restrict__ med_off,
                           const uint32_t* __restrict__ huge_off, int4* __restrict__ seg,
                           int4* __restrict__ med_rows, int4* __restrict__ huge_rows) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= m) return;
  const int b = row_ptr[v], e = row_ptr[v + 1];
  const int c = (e - b + kSplatSeg - 1) / kSplatSeg;
  const int s0 = (int)seg_off[v];
  const int slot0 = c > 1 ? (int)slot_off[v] : -1;
  for (int j = 0; j < c; ++j) {
    const int beg = b + j * kSplatSeg;
    seg[s0 + j] = make_int4((int)v, beg, min(beg + kSplatSeg, e), c > 1 ? slot0 + j : -1);
  }
  if (c > 1 && c <= kSplatMedSegs) med_rows[med_off[v]] = make_int4((int)v, slot0, c, 0);
  if (c > kSplatMedSegs) huge_rows[huge_off[v]] = make_int4((int)v, slot0, c, 0);
}

// Within each window of kSegWindow consecutive segments, order the segments by length,
// longest first (ties keep their order), so that the thread groups of a warp walk lists
// of similar length and finish together.  Windows keep the vertex order of the lattice
// at large, so the gathers of concurrently running warps stay local.  The splat's result
// does not depend on the order in which segments are processed.
constexpr int kSegWindow = 128;
__global__ void __launch_bounds__(kSegWindow) k_seg_window_sort(const int4* __restrict__ in,
                                                                int64_t nseg,
                                                                int4* __restrict__ out) {
  __shared__ int len[kSegWindow];
  const int64_t s = (int64_t)blockIdx.x * kSegWindow + threadIdx.x;
  const int4 sg = s < nseg ? in[s] : make_int4(0, 0, 0, 0);
  const int mine = s < nseg ? sg.z - sg.y : -1;
  len[threadIdx.x] = mine;
  __syncthreads();
  if (s >= nseg) return;
  int rank = 0;
  for (int j = 0; j < kSegWindow; ++j) {
    const int o = len[j];
    rank += (o > mine || (o == mine && j < (int)threadIdx.x)) ? 1 : 0;
  }
  out[(int64_t)blockIdx.x * kSegWindow + rank] = sg;
}

__global__ void k_iota(uint32_t* __restrict__ out, int64_t count) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p < count) out[p] = (uint32_t)p;
}

__global__ void k_row_ptr(const uint32_t* __restrict__ sorted_ids, int64_t nD, int64_t m,
                          int32_t* __restrict__ row_ptr) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p > nD) return;
  if (p == nD) {
    row_ptr[m] = (int32_t)nD;
    return;
  }
  const uint32_t v = sorted_ids[p];
  if (p == 0 || sorted_ids[p - 1] != v) row_ptr[v] = (int32_t)p;
}

// ---------------------------------------------------------------------------------
// Host orchestration.
// ---------------------------------------------------------------------------------
template <class T>
cudaError_t dalloc(T** p, size_t count, cudaStream_t st) {
  return dev_malloc((void**)p, std::max<size_t>(count, 1) * sizeof(T), st);
}

struct Temps {
  cudaStream_t st;
  std::vector<void*> ptrs;
  ~Temps() {
    for (void* p : ptrs) (void)cudaFreeAsync(p, st);
    clear_pending_error();
  }
  template <class T>
  cudaError_t get(T** p, size_t count) {
    cudaError_t e = dalloc(p, count, st);
    if (e == cudaSuccess) ptrs.push_back((void*)*p);
    return e;
  }
};

int bits_for(uint64_t v) {  // bits needed to hold values 0..v
  int b = 0;
  while (b < 64 && (v >> b) != 0) ++b;
  return b;
}

#define SGP_DISPATCH_D(D, KERNEL, GRID, BLOCK, ST, ...)                            \
  do {                                                                              \
    if ((D) <= 8) KERNEL<8><<<(GRID), (BLOCK), 0, (ST)>>>(__VA_ARGS__);             \
    else if ((D) <= 16) KERNEL<16><<<(GRID), (BLOCK), 0, (ST)>>>(__VA_ARGS__);      \
    else if ((D) <= 32) KERNEL<32><<<(GRID), (BLOCK), 0, (ST)>>>(__VA_ARGS__);      \
    else if ((D) <= 64) KERNEL<64><<<(GRID), (BLOCK), 0, (ST)>>>(__VA_ARGS__);      \
    else KERNEL<128><<<(GRID), (BLOCK), 0, (ST)>>>(__VA_ARGS__);                    \
    note_launches(1);                                                               \
  } while (0)

#define SGP_CHECK(expr, what)                                  \
  do {                                                         \
    cudaError_t e_ = (expr);                                   \
    if (e_ != cudaSuccess) return cuda_status(e_, what);       \
  } while (0)

}  // namespace

// Upload the hash multipliers to the current device once (blocking, so that every stream
// of the process sees them before its first build kernel).
static sgp_status ensure_coord_mults() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_status(e, "cudaGetDevice");
  if (dev < 0 || dev >= 64) {
    set_error("sgp_lattice_build: device ordinal out of range");
    return SGP_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (done[dev]) return SGP_OK;
  uint64_t table[kMaxD];
  for (int c = 0; c < kMaxD; ++c) table[c] = host_coord_mult(c);
  e = cudaMemcpyToSymbol(c_coord_mult, table, sizeof(table));
  if (e != cudaSuccess) return cuda_status(e, "uploading the hash multipliers");
  done[dev] = true;
  return SGP_OK;
}

sgp_status build_lattice(Lattice* L, const float* X, const float* ls) {
  cudaStream_t st = L->stream;
  {
    const sgp_status s0 = ensure_coord_mults();
    if (s0 != SGP_OK) return s0;
  }
  const int64_t n = L->n;
  const int d = L->d, D = L->D, r = L->r;
  const int64_t nD = n * D;
  Temps tmp{st, {}};

  // per-dimension factors of the elevation: scale / sqrt((j+1)(j+2)), scale = sqrt(d(d+1))/s
  const double scale = std::sqrt((double)(d * (d + 1))) / L->s;
  std::vector<double> hf(d);
  for (int j = 0; j < d; ++j) hf[j] = scale / std::sqrt((double)((j + 1) * (j + 2)));
  double* f = nullptr;
  SGP_CHECK(tmp.get(&f, d), "alloc f");
  SGP_CHECK(cudaMemcpyAsync(f, hf.data(), d * sizeof(double), cudaMemcpyHostToDevice, st),
            "copy f");

  int16_t* rem0 = nullptr;
  uint8_t* rank = nullptr;
  float* w_user = nullptr;
  int* qmm = nullptr;  // [2][D]: min, max of rem0 / D per coordinate
  SGP_CHECK(tmp.get(&rem0, nD), "alloc rem0");
  SGP_CHECK(tmp.get(&rank, nD), "alloc rank");
  SGP_CHECK(tmp.get(&w_user, nD), "alloc w");
  SGP_CHECK(tmp.get(&qmm, 2 * D), "alloc qmm");
  {
    std::vector<int> init(2 * D);
    for (int c = 0; c < D; ++c) {
      init[c] = 1 << 30;
      init[D + c] = -(1 << 30);
    }
    SGP_CHECK(cudaMemcpyAsync(qmm, init.data(), 2 * D * sizeof(int), cudaMemcpyHostToDevice, st),
              "copy qmm");
  }
  SGP_CHECK(cudaMemsetAsync(L->err, 0, sizeof(unsigned), st), "memset err");
  {
    const int B = 128;
    SGP_DISPATCH_D(D, k_elevate, (unsigned)ceil_div(n, B), B, st, X, ls, f, n, d, rem0, rank,
                   w_user, qmm, qmm + D, L->err, L->fault == FAULT_NAN_INPUT ? 1 : 0);
    SGP_CHECK(cudaGetLastError(), "k_elevate");
  }
  unsigned herr = 0;
  std::vector<int> hq(2 * D);
  SGP_CHECK(cudaMemcpyAsync(hq.data(), qmm, 2 * D * sizeof(int), cudaMemcpyDeviceToHost, st),
            "read qmm");
  SGP_CHECK(cudaMemcpyAsync(&herr, L->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st),
            "read err");
  SGP_CHECK(cudaStreamSynchronize(st), "sync elevate");
  if (herr & ERRBIT_NONFINITE) {
    set_error("sgp_lattice_build: X holds NaN/Inf or a lengthscale is not a finite positive");
    return SGP_ERR_NONFINITE;
  }
  if (herr & ERRBIT_RANGE) {
    set_error("sgp_lattice_build: a lattice coordinate exceeds the int16 key range "
              "(lengthscales too small for the spread of X)");
    return SGP_ERR_RANGE;
  }

  // 2. locality order
  CellPack pk{};
  {
    int used = 0;
    for (int c = 0; c < d && c < kMaxD; ++c) {
      const int b = bits_for((uint64_t)(hq[D + c] - hq[c]));
      if (used + b > 32) break;
      pk.ncoord = c + 1;
      pk.qmin[c] = hq[c];
      used += b;
      pk.shift[c] = b > 0 ? 32 - used : 0;  // a single-valued coordinate packs to 0
    }
    uint32_t *ka, *va, *kb, *vb, *rt;
    SGP_CHECK(tmp.get(&ka, n), "alloc sort");
    SGP_CHECK(tmp.get(&va, n), "alloc sort");
    SGP_CHECK(tmp.get(&kb, n), "alloc sort");
    SGP_CHECK(tmp.get(&vb, n), "alloc sort");
    SGP_CHECK(tmp.get(&rt, radix_temp_elems(n)), "alloc sort");
    k_point_key<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(rem0, n, D, pk, ka, va);
    note_launches(1);
    // the packed cell occupies the top `used` bits; bits below are zero
    const bool in_alt = used > 0 ? radix_sort_pairs(ka, va, kb, vb, n, 32, rt, st) : false;
    SGP_CHECK(dalloc(&L->perm, n, st), "alloc perm");
    SGP_CHECK(cudaMemcpyAsync(L->perm, in_alt ? vb : va, n * sizeof(int32_t),
                              cudaMemcpyDeviceToDevice, st),
              "copy perm");
    L->bytes += n * sizeof(int32_t);
  }

  // 3. hash insert
  uint64_t cap = 1024;
  if (L->fault != FAULT_HASH_FULL)  // SGP_FAULT=hash_full keeps the 1024-slot table
    while (cap < (uint64_t)(2 * nD)) cap <<= 1;
  const uint64_t mask = cap - 1;
  unsigned long long* table = nullptr;
  int32_t* entry_slot = nullptr;
  SGP_CHECK(tmp.get(&table, cap), "alloc hash table");
  SGP_CHECK(tmp.get(&entry_slot, nD), "alloc entry slots");
  SGP_CHECK(cudaMemsetAsync(table, 0xff, cap * sizeof(unsigned long long), st), "memset table");
  SGP_DISPATCH_D(D, k_insert, (unsigned)ceil_div(nD, 256), 256, st, L->perm, rem0, rank, nD, d,
                 table, mask, entry_slot, L->err);
  SGP_CHECK(cudaGetLastError(), "k_insert");

  // 4. numbering
  uint32_t *flags, *scan_tmp, *total;
  SGP_CHECK(tmp.get(&flags, nD), "alloc flags");
  SGP_CHECK(tmp.get(&scan_tmp, scan_temp_elems(nD)), "alloc scan");
  SGP_CHECK(tmp.get(&total, 1), "alloc total");
  k_owner_flags<<<(unsigned)ceil_div(nD, 256), 256, 0, st>>>(entry_slot, table, nD, flags);
  note_launches(1);
  exclusive_scan_u32(flags, nD, total, scan_tmp, st);
  uint32_t hm = 0;
  SGP_CHECK(cudaMemcpyAsync(&hm, total, sizeof(uint32_t), cudaMemcpyDeviceToHost, st), "read m");
  SGP_CHECK(cudaMemcpyAsync(&herr, L->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st),
            "read err");
  SGP_CHECK(cudaStreamSynchronize(st), "sync insert");
  if (herr & ERRBIT_HASH_FULL) {
    set_error("sgp_lattice_build: vertex hash table full");
    return SGP_ERR_HASH_FULL;
  }
  const int64_t m = hm;
  L->m = m;
  int32_t* slot_id = nullptr;
  SGP_CHECK(tmp.get(&slot_id, cap), "alloc slot ids");
  SGP_CHECK(dalloc(&L->keys, m * D, st), "alloc keys");
  L->bytes += m * D * sizeof(int16_t);
  uint64_t* vhash = nullptr;
  int2* vrange = nullptr;
  SGP_CHECK(tmp.get(&vhash, m), "alloc vertex hashes");
  SGP_CHECK(tmp.get(&vrange, m), "alloc vertex ranges");
  // vertex filter: about 8 bits per vertex, 2^16 .. 2^29 bits
  uint64_t bloom_bits = 1ull << 16;
  while (bloom_bits < 8ull * (uint64_t)m && bloom_bits < (1ull << 29)) bloom_bits <<= 1;
  uint32_t* bloom = nullptr;
  SGP_CHECK(tmp.get(&bloom, bloom_bits / 32), "alloc vertex filter");
  SGP_CHECK(cudaMemsetAsync(bloom, 0, bloom_bits / 8, st), "clear vertex filter");
  k_assign_ids<<<(unsigned)ceil_div(nD, 256), 256, 0, st>>>(flags, entry_slot, table, L->perm,
                                                           rem0, rank, nD, d, slot_id, L->keys,
                                                           vhash, vrange, bloom, bloom_bits - 1);
  note_launches(1);
  SGP_CHECK(dalloc(&L->idx, nD, st), "alloc idx");
  SGP_CHECK(dalloc(&L->w, nD, st), "alloc w");
  SGP_CHECK(dalloc(&L->rank, nD, st), "alloc rank");
  L->bytes += nD * (sizeof(int32_t) + sizeof(float) + sizeof(uint8_t));
  k_entry_ids<<<(unsigned)ceil_div(nD, 256), 256, 0, st>>>(entry_slot, slot_id, L->perm, w_user,
                                                          rank, nD, D, L->idx, L->w, L->rank);
  note_launches(1);
  SGP_CHECK(cudaGetLastError(), "numbering");

  // 5. neighbour table
  SGP_CHECK(dalloc(&L->nbr, (size_t)D * r * 2 * m, st), "alloc nbr");
  L->bytes += (size_t)D * r * 2 * m * sizeof(int32_t);
  unsigned long long* counts = nullptr;
  SGP_CHECK(tmp.get(&counts, 2 * D), "alloc counts");
  SGP_CHECK(cudaMemsetAsync(counts, 0, 2 * D * sizeof(unsigned long long), st), "clear counts");
  uint32_t* hasnb = nullptr;  // [ceil(D / 32)][m] neighbour bits per direction
  SGP_CHECK(tmp.get(&hasnb, (int64_t)((D + 31) / 32) * m), "alloc neighbour bits");
  {
    // sum_c A_c over the D coordinates, as the kernels compute A_c
    uint64_t sum_A = 0;
    for (int c = 0; c < D; ++c) sum_A += host_coord_mult(c);
    k_neighbours<<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(
        L->keys, vhash, vrange, m, d, r, sum_A, table, mask, slot_id, L->perm, rem0, rank,
        bloom, bloom_bits - 1, L->nbr, counts, hasnb);
    note_launches(1);
  }
  SGP_CHECK(cudaGetLastError(), "k_neighbours");

  // 6. splat lists: (vertex id, entry) sorted by id, stable in entry order
  {
    uint32_t *ka, *va, *kb, *vb, *rt;
    SGP_CHECK(tmp.get(&ka, nD), "alloc csr");
    SGP_CHECK(tmp.get(&va, nD), "alloc csr");
    SGP_CHECK(tmp.get(&kb, nD), "alloc csr");
    SGP_CHECK(tmp.get(&vb, nD), "alloc csr");
    SGP_CHECK(tmp.get(&rt, radix_temp_elems(nD)), "alloc csr");
    SGP_CHECK(cudaMemcpyAsync(ka, L->idx, nD * sizeof(uint32_t), cudaMemcpyDeviceToDevice, st),
              "copy ids");
    k_iota<<<(unsigned)ceil_div(nD, 256), 256, 0, st>>>(va, nD);
    note_launches(1);
    const int bits = std::max(1, bits_for((uint64_t)(m > 0 ? m - 1 : 0)));
    const bool in_alt = radix_sort_pairs(ka, va, kb, vb, nD, bits, rt, st);
    const uint32_t* sorted_ids = in_alt ? kb : ka;
    const uint32_t* sorted_entries = in_alt ? vb : va;
    SGP_CHECK(dalloc(&L->items, nD, st), "alloc items");
    SGP_CHECK(dalloc(&L->row_ptr, m + 1, st), "alloc row_ptr");
    L->bytes += nD * sizeof(int2) + (m + 1) * sizeof(int32_t);
    k_splat_items<<<(unsigned)ceil_div(nD, 256), 256, 0, st>>>(sorted_entries, L->w, nD, D,
                                                              L->items);
    note_launches(1);
    k_row_ptr<<<(unsigned)ceil_div(nD + 1, 256), 256, 0, st>>>(sorted_ids, nD, m, L->row_ptr);
    note_launches(1);
    SGP_CHECK(cudaGetLastError(), "splat lists");
  }

  // 7. splat segments (load balance)
  {
    uint32_t *cnt, *slots, *med, *huge, *tot, *stmp;
    SGP_CHECK(tmp.get(&cnt, m), "alloc seg");
    SGP_CHECK(tmp.get(&slots, m), "alloc seg");
    SGP_CHECK(tmp.get(&med, m), "alloc seg");
    SGP_CHECK(tmp.get(&huge, m), "alloc seg");
    SGP_CHECK(tmp.get(&tot, 4), "alloc seg");
    SGP_CHECK(tmp.get(&stmp, scan_temp_elems(m)), "alloc seg");
    k_seg_count<<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(L->row_ptr, m, cnt, slots, med, huge);
    note_launches(1);
    exclusive_scan_u32(cnt, m, tot + 0, stmp, st);
    exclusive_scan_u32(slots, m, tot + 1, stmp, st);
    exclusive_scan_u32(med, m, tot + 2, stmp, st);
    exclusive_scan_u32(huge, m, tot + 3, stmp, st);
    uint32_t ht[4];
    SGP_CHECK(cudaMemcpyAsync(ht, tot, sizeof(ht), cudaMemcpyDeviceToHost, st), "read seg");
    SGP_CHECK(cudaStreamSynchronize(st), "sync seg");
    L->nseg = ht[0];
    L->nslots = ht[1];
    L->nmed = ht[2];
    L->nhuge = ht[3];
    SGP_CHECK(dalloc(&L->seg, L->nseg, st), "alloc seg");
    SGP_CHECK(dalloc(&L->med_rows, L->nmed, st), "alloc seg");
    SGP_CHECK(dalloc(&L->huge_rows, L->nhuge, st), "alloc seg");
    L->bytes += (L->nseg + L->nmed + L->nhuge) * sizeof(int4);
    int4* seg_unsorted = nullptr;
    SGP_CHECK(tmp.get(&seg_unsorted, std::max<int64_t>(L->nseg, 1)), "alloc seg");
    k_seg_fill<<<(unsigned)ceil_div(m, 256), 256, 0, st>>>(L->row_ptr, m, cnt, slots, med, huge,
                                                          seg_unsorted, L->med_rows,
                                                          L->huge_rows);
    if (L->nseg > 0)
      k_seg_window_sort<<<(unsigned)ceil_div(L->nseg, kSegWindow), kSegWindow, 0, st>>>(
          seg_unsorted, L->nseg, L->seg);
    note_launches(2);
    SGP_CHECK(cudaGetLastError(), "splat segments");
  }
  // 8. direction lists of a sparse lattice (counts from k_neighbours)
  {
    std::vector<unsigned long long> hc(D);
    SGP_CHECK(cudaMemcpyAsync(hc.data(), counts, D * sizeof(unsigned long long),
                              cudaMemcpyDeviceToHost, st),
              "read counts");
    SGP_CHECK(cudaStreamSynchronize(st), "sync counts");
    int64_t total = 0, largest = 0;
    for (int j = 0; j < D; ++j) {
      total += (int64_t)hc[j];
      largest = std::max<int64_t>(largest, (int64_t)hc[j]);
    }
    if (m > 0 && (double)total <= kSparseFrac * (double)D * (double)m) {
      L->sparse = true;
      L->act_max = largest;
      L->act_off.assign(D + 1, 0);
      for (int j = 0; j < D; ++j) L->act_off[j + 1] = L->act_off[j] + (int64_t)hc[j];
      SGP_CHECK(dalloc(&L->act, std::max<int64_t>(total, 1), st), "alloc direction lists");
      SGP_CHECK(dalloc(&L->epoch, m, st), "alloc epochs");
      L->bytes += (size_t)total * sizeof(int32_t) + (size_t)m * sizeof(int32_t);
      SGP_CHECK(dalloc(&L->act_off_dev, D + 1, st), "alloc list offsets");
      SGP_CHECK(cudaMemcpyAsync(L->act_off_dev, L->act_off.data(), (D + 1) * sizeof(int64_t),
                                cudaMemcpyHostToDevice, st),
                "copy list offsets");
      k_active_fill<<<(unsigned)ceil_div(m, kFillThreads), kFillThreads, 0, st>>>(
          hasnb, m, D, L->act_off_dev, counts + D, L->act);
      note_launches(1);
      // powers of the symmetric blur's centre tap g_0 (stored rows are rescaled lazily)
      std::vector<float> pw(2 * D + 1);
      for (int q = 0; q <= 2 * D; ++q) pw[q] = (float)std::pow(L->half[0], (double)q);
      SGP_CHECK(dalloc(&L->g0pow, 2 * D + 1, st), "alloc tap powers");
      SGP_CHECK(cudaMemcpyAsync(L->g0pow, pw.data(), pw.size() * sizeof(float),
                                cudaMemcpyHostToDevice, st),
                "copy tap powers");
      SGP_CHECK(cudaGetLastError(), "direction lists");
    }
  }
  SGP_CHECK(cudaStreamSynchronize(st), "sync build");
  return SGP_OK;
}

}  // namespace sgp
