// Device primitives: exclusive prefix sum and a stable LSD radix sort.
//
// These back the memory-pool sizing (exclusive scans of per-rule sizes, the
// "memory pool" of Section IV-B), the edge deduplication at load time and the
// canonical ordering of every result.
#include <type_traits>

#include "gt_device.cuh"

namespace gt {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 8;
constexpr int kScanChunk = kScanThreads * kScanItems;

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += t;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the block
// total through *total.
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t* total) {
  __shared__ int64_t warp_sums[kScanThreads / 32 + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = warp_incl_scan(v);
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < kScanThreads / 32 ? warp_sums[lane] : 0;
    int64_t wi = warp_incl_scan(w);
    if (lane < kScanThreads / 32) warp_sums[lane] = wi - w;
    if (lane == kScanThreads / 32 - 1) warp_sums[kScanThreads / 32] = wi;  // slot after the last warp
  }
  __syncthreads();
  int64_t r = warp_sums[warp] + incl - v;
  if (total) *total = warp_sums[kScanThreads / 32];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(const int64_t* __restrict__ in, int64_t n,
                                                                   int64_t* __restrict__ bsum) {
  const int64_t base = int64_t(blockIdx.x) * kScanChunk;
  int64_t s = 0;
  for (int i = threadIdx.x; i < kScanChunk; i += kScanThreads) {
    int64_t idx = base + i;
    if (idx < n) s += in[idx];
  }
  int64_t total;
  block_excl_scan(s, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_apply_kernel(const int64_t* in, int64_t* out, int64_t n,
                                                                  const int64_t* __restrict__ boff) {
  __shared__ int64_t tile[kScanChunk];
  const int64_t base = int64_t(blockIdx.x) * kScanChunk;
  for (int i = threadIdx.x; i < kScanChunk; i += kScanThreads) {
    int64_t idx = base + i;
    tile[i] = idx < n ? in[idx] : 0;
  }
  __syncthreads();
  int64_t local[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    local[j] = tile[threadIdx.x * kScanItems + j];
    s += local[j];
  }
  int64_t off = block_excl_scan(s, nullptr) + (boff ? boff[blockIdx.x] : 0);
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    tile[threadIdx.x * kScanItems + j] = off;
    off += local[j];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kScanChunk; i += kScanThreads) {
    int64_t idx = base + i;
    if (idx < n) out[idx] = tile[i];
  }
}

// ---- radix sort -------------------------------------------------------------

constexpr int kRsThreads = 256;  // one thread per digit value in the per-tile bookkeeping
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsItems = 8;      // keys per thread by default ("radix_items" 16 doubles the tile)
constexpr int kRsTile = kRsThreads * kRsItems;  // keys per tile (the smallest tile: scratch is sized for it)

// Per-tile digit counts, stored tile-major (hist[tile * 256 + d]) so that
// each CTA writes one contiguous row.
template <int ITEMS>
__global__ void __launch_bounds__(kRsThreads) radix_upsweep_kernel(const uint64_t* __restrict__ keys, int64_t n,
                                                                   int shift, uint32_t mask,
                                                                   uint32_t* __restrict__ hist) {
  constexpr int kRsItems = ITEMS, kRsTile = kRsThreads * ITEMS;
  __shared__ uint32_t h[kRsWarps][256];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t wbase = int64_t(blockIdx.x) * kRsTile + int64_t(warp) * 32 * kRsItems;
  uint64_t key[kRsItems];  // every load issued before the counters are cleared
#pragma unroll
  for (int it = 0; it < kRsItems; ++it) {
    const int64_t idx = wbase + it * 32 + lane;
    key[it] = idx < n ? keys[idx] : 0;
  }
  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) h[i / 256][i % 256] = 0;
  __syncthreads();
  // counting only: one shared atomic per key into the warp's own counters
  // (measured faster than ballot multisplit, also when all keys share a digit)
#pragma unroll
  for (int it = 0; it < kRsItems; ++it) {
    const int64_t idx = wbase + it * 32 + lane;
    if (idx < n) atomicAdd(&h[warp][uint32_t(key[it] >> shift) & mask], 1u);
  }
  __syncthreads();
  const int d = threadIdx.x;
  uint32_t t = 0;
#pragma unroll
  for (int w = 0; w < kRsWarps; ++w) t += h[w][d];
  hist[int64_t(blockIdx.x) * 256 + d] = t;
}

// Output offsets of every (tile, digit): offs[tile * 256 + d] = (keys of
// smaller digits) + (keys of digit d in earlier tiles).  Tiles are grouped in
// chunks of kRsChunk: per-chunk digit sums (digit-major, so one scan orders
// them by digit, then chunk), then a running sum inside each chunk.
constexpr int kRsChunk = 64;

__global__ void __launch_bounds__(256) radix_chunk_sum_kernel(const uint32_t* __restrict__ hist, int64_t ntiles,
                                                               int64_t nchunks, int64_t* __restrict__ csum) {
  const int64_t c = blockIdx.x;
  const int d = threadIdx.x;
  const int64_t t1 = min(ntiles, (c + 1) * kRsChunk);
  int64_t sum = 0;
  for (int64_t t = c * kRsChunk; t < t1; ++t) sum += hist[t * 256 + d];
  csum[int64_t(d) * nchunks + c] = sum;
}

__global__ void __launch_bounds__(256) radix_chunk_offsets_kernel(const uint32_t* __restrict__ hist,
                                                                   const int64_t* __restrict__ cpre, int64_t ntiles,
                                                                   int64_t nchunks, int64_t* __restrict__ offs) {
  const int64_t c = blockIdx.x;
  const int d = threadIdx.x;
  const int64_t t1 = min(ntiles, (c + 1) * kRsChunk);
  int64_t run = cpre[int64_t(d) * nchunks + c];
  for (int64_t t = c * kRsChunk; t < t1; ++t) {
    offs[t * 256 + d] = run;
    run += hist[t * 256 + d];
  }
}

// Stable scatter of one tile.  Warp w owns the w-th slice of the tile and
// ranks its keys 32 at a time in lane order; per-digit counts across warps
// and digits give every key its place in the tile sorted by digit.  The tile
// is rearranged in shared memory in that order and written out with
// consecutive threads writing consecutive addresses of each digit's run.
template <int VB, int ITEMS>
__global__ void __launch_bounds__(kRsThreads, ITEMS == 8 ? 4 : 2) radix_downsweep_kernel(
    const uint64_t* __restrict__ kin, uint64_t* __restrict__ kout, const void* __restrict__ vin,
    void* __restrict__ vout, int64_t n, int shift, uint32_t mask, const int64_t* __restrict__ offs) {
  constexpr int kRsItems = ITEMS, kRsTile = kRsThreads * ITEMS;
  __shared__ uint32_t wcnt[kRsWarps][256];
  __shared__ uint32_t dstart[256];
  __shared__ uint32_t wsum[kRsWarps];
  __shared__ int64_t goff[256];
  extern __shared__ __align__(16) unsigned char rs_smem[];
  uint64_t* skey = reinterpret_cast<uint64_t*>(rs_smem);
  unsigned char* sval = rs_smem + kRsTile * 8;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t tbase = int64_t(blockIdx.x) * kRsTile;
  const int64_t wbase = tbase + int64_t(warp) * 32 * kRsItems;
  using VT = typename std::conditional<VB == 8, uint64_t, uint32_t>::type;
  uint64_t key[kRsItems];
  uint32_t rank[kRsItems];
  VT val[kRsItems];
  // the tile's keys and values and this digit's output offset are all
  // requested before the first barrier, so one memory round trip starts a tile
#pragma unroll
  for (int it = 0; it < kRsItems; ++it) {
    const int64_t idx = wbase + it * 32 + lane;
    const bool valid = idx < n;
    key[it] = valid ? kin[idx] : 0;
    val[it] = 0;
    if (VB != 0 && valid) val[it] = static_cast<const VT*>(vin)[idx];
  }
  goff[threadIdx.x] = offs[int64_t(blockIdx.x) * 256 + threadIdx.x];
  for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) wcnt[i / 256][i % 256] = 0;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kRsItems; ++it) {
    const int64_t idx = wbase + it * 32 + lane;
    const bool valid = idx < n;
    const uint32_t d = uint32_t(key[it] >> shift) & mask;
    const unsigned peers = warp_digit_peers(d, __ballot_sync(0xffffffffu, valid));
    const uint32_t before = wcnt[warp][d];
    const uint32_t r = __popc(peers & lt_mask);
    rank[it] = before + r;
    __syncwarp();
    if (valid && r == 0) wcnt[warp][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per digit: exclusive prefix over warps, then exclusive prefix over digits
  const int dd = threadIdx.x;
  uint32_t run = 0;
#pragma unroll
  for (int w = 0; w < kRsWarps; ++w) {
    const uint32_t c = wcnt[w][dd];
    wcnt[w][dd] = run;
    run += c;
  }
  uint32_t incl = run;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t wpre = 0;
#pragma unroll
  for (int w = 0; w < kRsWarps; ++w) wpre += w < warp ? wsum[w] : 0u;
  dstart[dd] = wpre + incl - run;
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kRsItems; ++it) {
    const int64_t idx = wbase + it * 32 + lane;
    if (idx < n) {
      const uint32_t d = uint32_t(key[it] >> shift) & mask;
      const uint32_t lp = dstart[d] + wcnt[warp][d] + rank[it];
      skey[lp] = key[it];
      if (VB != 0) reinterpret_cast<VT*>(sval)[lp] = val[it];
    }
  }
  __syncthreads();
  const int tn = int(n - tbase < kRsTile ? n - tbase : kRsTile);
#pragma unroll
  for (int it = 0; it < kRsItems; ++it) {
    const int i = it * kRsThreads + threadIdx.x;
    if (i < tn) {
      const uint64_t k = skey[i];
      const uint32_t d = uint32_t(k >> shift) & mask;
      const int64_t pos = goff[d] + (i - int64_t(dstart[d]));
      kout[pos] = k;
      if (VB != 0) static_cast<VT*>(vout)[pos] = reinterpret_cast<const VT*>(sval)[i];
    }
  }
}

// The same scatter as a persistent kernel (one CTA per tile slot of the
// SMs) that copies the next full tile's keys and values into shared memory
// with asynchronous 16-byte copies while it ranks and scatters the current
// one; the tile it has just ranked is staged in place.  Same results (the
// ranking order and the offsets are the same).  Needs 16-byte-aligned key and
// value arrays; the caller checks.
template <int VB>
__global__ void __launch_bounds__(kRsThreads, 3) radix_scatter_pf_kernel(
    const uint64_t* __restrict__ kin, uint64_t* __restrict__ kout, const void* __restrict__ vin,
    void* __restrict__ vout, int64_t n, int shift, uint32_t mask, const int64_t* __restrict__ offs, int64_t ntiles) {
  constexpr int kRsItems = 8, kRsTile = kRsThreads * 8;
  constexpr int kBuf = kRsTile * (8 + VB);  // bytes of one tile (keys, then values)
  __shared__ uint32_t wcnt[kRsWarps][256];
  __shared__ uint32_t dstart[256];
  __shared__ uint32_t wsum[kRsWarps];
  __shared__ int64_t goff[256];
  extern __shared__ __align__(16) unsigned char rs_smem[];  // two tile buffers
  using VT = typename std::conditional<VB == 8, uint64_t, uint32_t>::type;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int64_t nfull = n / kRsTile;  // tiles copied asynchronously; the last partial one is read directly
  auto prefetch = [&](int64_t t, unsigned char* buf) {
    if (t >= nfull) return;
    const unsigned char* gk = reinterpret_cast<const unsigned char*>(kin + t * kRsTile);
    const unsigned char* gv = static_cast<const unsigned char*>(vin) + t * kRsTile * VB;
    for (int c = threadIdx.x; c < kBuf / 16; c += kRsThreads) {
      const unsigned char* src = c < kRsTile * 8 / 16 ? gk + 16 * c : gv + 16 * (c - kRsTile * 8 / 16);
      const unsigned dst = unsigned(__cvta_generic_to_shared(buf + 16 * c));
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
  };
  int b = 0;
  prefetch(blockIdx.x, rs_smem);
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, b ^= 1) {
    unsigned char* cur = rs_smem + b * kBuf;
    prefetch(t + gridDim.x, rs_smem + (b ^ 1) * kBuf);  // into the buffer the previous tile staged in
    asm volatile("cp.async.commit_group;" ::: "memory");
    asm volatile("cp.async.wait_group 1;" ::: "memory");  // this tile's copies are done
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) wcnt[i / 256][i % 256] = 0;
    goff[threadIdx.x] = offs[t * 256 + threadIdx.x];
    __syncthreads();
    const int64_t tbase = t * kRsTile;
    const bool staged = t < nfull;
    const uint64_t* sk_in = reinterpret_cast<const uint64_t*>(cur);
    const VT* sv_in = reinterpret_cast<const VT*>(cur + kRsTile * 8);
    uint64_t key[kRsItems];
    uint32_t rank[kRsItems];
    VT val[kRsItems];
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
      const int j = warp * 32 * kRsItems + it * 32 + lane;  // the same item order as the one-tile kernel
      const bool valid = tbase + j < n;
      key[it] = staged ? sk_in[j] : (valid ? kin[tbase + j] : 0);
      val[it] = 0;
      if (VB != 0 && valid) val[it] = staged ? sv_in[j] : static_cast<const VT*>(vin)[tbase + j];
      const uint32_t d = uint32_t(key[it] >> shift) & mask;
      const unsigned peers = warp_digit_peers(d, __ballot_sync(0xffffffffu, valid));
      const uint32_t before = wcnt[warp][d];
      const uint32_t r = __popc(peers & lt_mask);
      rank[it] = before + r;
      __syncwarp();
      if (valid && r == 0) wcnt[warp][d] = before + __popc(peers);
      __syncwarp();
    }
    __syncthreads();  // also: the tile's buffer is read, it becomes the staging area
    const int dd = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) {
      const uint32_t c = wcnt[w][dd];
      wcnt[w][dd] = run;
      run += c;
    }
    uint32_t incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t wpre = 0;
#pragma unroll
    for (int w = 0; w < kRsWarps; ++w) wpre += w < warp ? wsum[w] : 0u;
    dstart[dd] = wpre + incl - run;
    __syncthreads();
    uint64_t* skey = reinterpret_cast<uint64_t*>(cur);
    VT* sval = reinterpret_cast<VT*>(cur + kRsTile * 8);
#pragma unroll
    for (int it = 0; it < kRsItems; ++it) {
      const int j = warp * 32 * kRsItems + it * 32 + lane;
      if (tbase + j < n) {
        const uint32_t d = uint32_t(key[it] >> shift) & mask;
        const uint32_t lp = dstart[d] + wcnt[warp][d] + rank[it];
        skey[lp] = key[it];
        if (VB != 0) sval[lp] = val[it];
      }
    }
    __syncthreads();
    const int tn = int(n - tbase < kRsTile ? n - tbase : kRsTile);
    for (int i = threadIdx.x; i < tn; i += kRsThreads) {
      const uint64_t k = skey[i];
      const uint32_t d = uint32_t(k >> shift) & mask;
      const int64_t pos = goff[d] + (i - int64_t(dstart[d]));
      kout[pos] = k;
      if (VB != 0) static_cast<VT*>(vout)[pos] = sval[i];
    }
    __syncthreads();  // the staging buffer is read before the next prefetch lands in it
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int VB, int ITEMS>
void launch_downsweep(const uint64_t* ka, uint64_t* kb, const void* va, void* vb, int64_t n, int shift, uint32_t mask,
                      int64_t ntiles, const int64_t* offs, cudaStream_t s) {
  const bool aligned = (reinterpret_cast<uintptr_t>(ka) & 15) == 0 && (reinterpret_cast<uintptr_t>(va) & 15) == 0;
  if (ITEMS == 8 && aligned && t_call_ctx && t_call_ctx->param("radix_prefetch", 0) != 0) {
    constexpr size_t smem2 = size_t(2) * kRsTile * (8 + VB);
    GT_CUDA(cudaFuncSetAttribute(radix_scatter_pf_kernel<VB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 int(smem2)));
    const int64_t grid = std::min<int64_t>(ntiles, int64_t(t_call_ctx->num_sms) * 3);
    Phase ph(t_call_ctx, "radix_pass", s);
    radix_scatter_pf_kernel<VB><<<unsigned(grid), kRsThreads, smem2, s>>>(ka, kb, va, vb, n, shift, mask, offs,
                                                                          ntiles);
    GT_LAUNCH_CHECK();
    return;
  }
  constexpr size_t smem = size_t(kRsThreads) * ITEMS * (8 + VB);
  GT_CUDA(cudaFuncSetAttribute(radix_downsweep_kernel<VB, ITEMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               int(smem)));
  Phase ph(t_call_ctx, "radix_pass", s);  // one span per scatter pass
  radix_downsweep_kernel<VB, ITEMS><<<unsigned(ntiles), kRsThreads, smem, s>>>(ka, kb, va, vb, n, shift, mask, offs);
  GT_LAUNCH_CHECK();
}

template <int ITEMS>
void radix_passes(uint64_t* ka, uint64_t* kb, void* va, void* vb, int value_bytes, int64_t n, const int* pass_shift,
                  const int* pass_bits, int npass, void* scratch, cudaStream_t s, bool& swapped) {
  constexpr int tile = kRsThreads * ITEMS;
  const int64_t ntiles = (n + tile - 1) / tile;
  const int64_t nchunks = (ntiles + kRsChunk - 1) / kRsChunk;
  const int64_t m = 256 * ntiles, mc = 256 * nchunks;
  uint32_t* hist = static_cast<uint32_t*>(scratch);
  int64_t* offs = reinterpret_cast<int64_t*>(static_cast<char*>(scratch) + ((size_t(m) * 4 + 15) / 16 * 16));
  int64_t* csum = offs + m;
  int64_t* cpre = csum + mc;
  void* sscratch = cpre + mc;
  swapped = false;
  for (int p = 0; p < npass; ++p) {
    const int shift = pass_shift[p];
    const uint32_t mask = (1u << pass_bits[p]) - 1u;
    radix_upsweep_kernel<ITEMS><<<unsigned(ntiles), kRsThreads, 0, s>>>(ka, n, shift, mask, hist);
    GT_LAUNCH_CHECK();
    radix_chunk_sum_kernel<<<unsigned(nchunks), 256, 0, s>>>(hist, ntiles, nchunks, csum);
    GT_LAUNCH_CHECK();
    exclusive_scan_i64(csum, cpre, mc, sscratch, s);
    radix_chunk_offsets_kernel<<<unsigned(nchunks), 256, 0, s>>>(hist, cpre, ntiles, nchunks, offs);
    GT_LAUNCH_CHECK();
    if (value_bytes == 4)
      launch_downsweep<4, ITEMS>(ka, kb, va, vb, n, shift, mask, ntiles, offs, s);
    else if (value_bytes == 8)
      launch_downsweep<8, ITEMS>(ka, kb, va, vb, n, shift, mask, ntiles, offs, s);
    else
      launch_downsweep<0, ITEMS>(ka, kb, nullptr, nullptr, n, shift, mask, ntiles, offs, s);
    std::swap(ka, kb);
    std::swap(va, vb);
    swapped = !swapped;
  }
}

}  // namespace

size_t scan_scratch_bytes(int64_t n) {
  int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  if (nb <= 1) return 0;
  return size_t(2 * nb) * sizeof(int64_t) + scan_scratch_bytes(nb);
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, void* scratch, cudaStream_t s) {
  if (n <= 0) return;
  int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  if (nb == 1) {
    scan_apply_kernel<<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    GT_LAUNCH_CHECK();
    return;
  }
  int64_t* bsum = static_cast<int64_t*>(scratch);
  int64_t* boff = bsum + nb;
  scan_reduce_kernel<<<unsigned(nb), kScanThreads, 0, s>>>(in, n, bsum);
  GT_LAUNCH_CHECK();
  exclusive_scan_i64(bsum, boff, nb, boff + nb, s);
  scan_apply_kernel<<<unsigned(nb), kScanThreads, 0, s>>>(in, out, n, boff);
  GT_LAUNCH_CHECK();
}

size_t radix_scratch_bytes(int64_t n, bool, int) {
  const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
  const int64_t nchunks = (ntiles + kRsChunk - 1) / kRsChunk;
  const int64_t m = 256 * ntiles, mc = 256 * nchunks;
  return size_t(m) * 4 + size_t(m) * 8 + size_t(2 * mc) * 8 + scan_scratch_bytes(mc) + 256;
}

void radix_sort_u64(uint64_t* keys_in, uint64_t* keys_out, void* vals_in, void* vals_out, int value_bytes,
                    int64_t n, int begin_bit, int end_bit, void* scratch, cudaStream_t s) {
  radix_sort_u64_split(keys_in, keys_out, vals_in, vals_out, value_bytes, n, begin_bit, end_bit, end_bit, end_bit,
                       scratch, s);
}

void radix_sort_u64_split(uint64_t* keys_in, uint64_t* keys_out, void* vals_in, void* vals_out, int value_bytes,
                          int64_t n, int begin_a, int end_a, int begin_b, int end_b, void* scratch, cudaStream_t s) {
  if (n <= 0) return;
  // digit passes: [begin_a, end_a) then [begin_b, end_b), 8 bits at a time
  int pass_shift[16], pass_bits[16], npass = 0;
  for (int r = 0; r < 2; ++r) {
    const int lo = r ? begin_b : begin_a, hi = r ? end_b : end_a;
    for (int shift = lo; shift < hi && npass < 16; shift += 8) {
      pass_shift[npass] = shift;
      pass_bits[npass++] = hi - shift < 8 ? hi - shift : 8;
    }
  }
  // digit passes over tiles of 2048 keys, or 4096 with "radix_items" 16
  const int items = t_call_ctx ? int(t_call_ctx->param("radix_items", kRsItems)) : kRsItems;
  bool swapped = false;
  if (items == 16)
    radix_passes<16>(keys_in, keys_out, vals_in, vals_out, value_bytes, n, pass_shift, pass_bits, npass, scratch, s,
                     swapped);
  else
    radix_passes<8>(keys_in, keys_out, vals_in, vals_out, value_bytes, n, pass_shift, pass_bits, npass, scratch, s,
                    swapped);
  uint64_t* ka = swapped ? keys_out : keys_in;
  void* va = swapped ? vals_out : vals_in;
  // after the loop the sorted data is in ka / va
  if (ka != keys_out) {
    GT_CUDA(cudaMemcpyAsync(keys_out, ka, size_t(n) * 8, cudaMemcpyDeviceToDevice, s));
    if (value_bytes)
      GT_CUDA(cudaMemcpyAsync(vals_out, va, size_t(n) * value_bytes, cudaMemcpyDeviceToDevice, s));
  }
}

}  // namespace gt
