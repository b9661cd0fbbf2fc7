// Device-wide exclusive scan and stable LSD radix sort, used while numbering lattice
// vertices and grouping point/vertex incidences by vertex during the build.
#include "sgp_internal.cuh"

namespace sgp {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortBatches = 8;                       // 32-item batches per warp
constexpr int kSortTile = kSortThreads * kSortBatches;  // 2048 items per block

// Exclusive block scan of one value per thread; returns the block total in *total.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[32];
  __shared__ uint32_t block_total;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  const int nwarps = blockDim.x >> 5;
  if (warp == 0) {
    uint32_t s = lane < nwarps ? warp_sums[lane] : 0u;
    uint32_t si = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, si, o);
      if (lane >= o) si += t;
    }
    if (lane < nwarps) warp_sums[lane] = si - s;
    if (lane == 31) block_total = si;  // nwarps <= 32
  }
  __syncthreads();
  const uint32_t res = warp_sums[warp] + inc - v;
  if (total) *total = block_total;
  __syncthreads();
  return res;
}

__global__ void k_scan_reduce(const uint32_t* __restrict__ data, int64_t n,
                              uint32_t* __restrict__ block_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += data[base + i];
  uint32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = total;
}

__global__ void k_scan_top(uint32_t* __restrict__ block_sums, int64_t nb,
                           uint32_t* __restrict__ total_out) {
  uint32_t carry = 0;
  for (int64_t base = 0; base < nb; base += kScanTile) {
    const int64_t my = base + (int64_t)threadIdx.x * kScanItems;
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      v[i] = (my + i < nb) ? block_sums[my + i] : 0u;
      s += v[i];
    }
    uint32_t tile_total;
    uint32_t run = carry + block_exclusive_scan(s, &tile_total);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
      if (my + i < nb) block_sums[my + i] = run;
      run += v[i];
    }
    carry += tile_total;
  }
  if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void k_scan_down(uint32_t* __restrict__ data, int64_t n,
                            const uint32_t* __restrict__ block_sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? data[base + i] : 0u;
    s += v[i];
  }
  uint32_t run = block_sums[blockIdx.x] + block_exclusive_scan(s, nullptr);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) data[base + i] = run;
    run += v[i];
  }
}

__global__ void k_radix_hist(const uint32_t* __restrict__ keys, int64_t n, int shift,
                             uint32_t* __restrict__ hist, int64_t nblk) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
    const int64_t e = base + i;
    if (e < n) atomicAdd(&h[(keys[e] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter: each warp owns a contiguous run of kSortBatches*32 items and walks it
// in order; lanes holding the same digit are ranked by lane within a batch.
__global__ void k_radix_scatter(const uint32_t* __restrict__ kin,
                                const uint32_t* __restrict__ vin, uint32_t* __restrict__ kout,
                                uint32_t* __restrict__ vout, int64_t n, int shift,
                                const uint32_t* __restrict__ offs, int64_t nblk) {
  __shared__ uint32_t cnt[kSortWarps][256];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * kSortTile + (int64_t)warp * (kSortBatches * 32);
  for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&cnt[0][0])[i] = 0u;
  __syncthreads();
  for (int b = 0; b < kSortBatches; ++b) {
    const int64_t e = base + b * 32 + lane;
    const bool valid = e < n;
    const uint32_t dig = valid ? ((kin[e] >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, dig);
    if (valid && lane == __ffs(peers) - 1) cnt[warp][dig] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    const int dig = threadIdx.x;
    uint32_t run = offs[(int64_t)dig * nblk + blockIdx.x];
    for (int w = 0; w < kSortWarps; ++w) {
      const uint32_t c = cnt[w][dig];
      cnt[w][dig] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int b = 0; b < kSortBatches; ++b) {
    const int64_t e = base + b * 32 + lane;
    const bool valid = e < n;
    const uint32_t key = valid ? kin[e] : 0u;
    const uint32_t dig = valid ? ((key >> shift) & 255u) : 256u;
    const unsigned peers = __match_any_sync(0xffffffffu, dig);
    const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    const uint32_t pos = valid ? cnt[warp][dig] + rank : 0u;
    if (valid) {
      kout[pos] = key;
      vout[pos] = vin[e];
    }
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) cnt[warp][dig] += __popc(peers);
    __syncwarp();
  }
}

}  // namespace

size_t scan_temp_elems(int64_t n) { return (size_t)ceil_div(n > 0 ? n : 1, kScanTile); }

void exclusive_scan_u32(uint32_t* data, int64_t n, uint32_t* total, uint32_t* tmp,
                        cudaStream_t st) {
  if (n <= 0) {
    if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), st);
    return;
  }
  const int64_t nb = ceil_div(n, kScanTile);
  k_scan_reduce<<<(unsigned)nb, kScanThreads, 0, st>>>(data, n, tmp);
  k_scan_top<<<1, kScanThreads, 0, st>>>(tmp, nb, total);
  k_scan_down<<<(unsigned)nb, kScanThreads, 0, st>>>(data, n, tmp);
  note_launches(3);
}

size_t radix_temp_elems(int64_t n) {
  const int64_t nblk = ceil_div(n > 0 ? n : 1, kSortTile);
  return (size_t)(256 * nblk) + scan_temp_elems(256 * nblk);
}

bool radix_sort_pairs(uint32_t* keys, uint32_t* vals, uint32_t* keys_alt, uint32_t* vals_alt,
                      int64_t n, int bits, uint32_t* tmp, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return false;
  const int64_t nblk = ceil_div(n, kSortTile);
  uint32_t* hist = tmp;
  uint32_t* scan_tmp = tmp + 256 * nblk;
  bool alt = false;
  for (int shift = 0; shift < bits; shift += 8) {
    const uint32_t* kin = alt ? keys_alt : keys;
    const uint32_t* vin = alt ? vals_alt : vals;
    uint32_t* kout = alt ? keys : keys_alt;
    uint32_t* vout = alt ? vals : vals_alt;
    k_radix_hist<<<(unsigned)nblk, kSortThreads, 0, st>>>(kin, n, shift, hist, nblk);
    exclusive_scan_u32(hist, 256 * nblk, nullptr, scan_tmp, st);
    k_radix_scatter<<<(unsigned)nblk, kSortThreads, 0, st>>>(kin, vin, kout, vout, n, shift,
                                                            hist, nblk);
    note_launches(2);
    alt = !alt;
  }
  return alt;
}

}  // namespace sgp
