// Stable LSD radix sort (8-bit digits) and exclusive scans.
//
// Tile = 256 threads x 8 rounds of 32 keys = 2048 keys.  Within a tile each
// warp owns 256 consecutive keys and ranks them round by round: lanes with
// the same digit are found with __match_any_sync, a lane's rank is the
// number of equal-digit lanes before it plus the warp's running count of
// that digit (kept in shared memory), which preserves input order.  Per-
// warp counts are then prefix-summed across the 8 warps, and a tile's
// global offset for a digit comes from the digit-major scan of all tiles'
// histograms.  Inputs of up to SMALL_N keys are sorted by one CTA that
// walks its tiles in order (one launch for all passes).  A sort whose count
// only the device knows launches that CTA and one cooperative kernel that
// runs every multi-CTA pass when the count is larger; the segments of a
// batch can be sorted one CTA each.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace hfcr {

namespace {

constexpr int TPB = 256;
constexpr int ROUNDS = 8;
constexpr int TILE = TPB * ROUNDS;  // 2048
constexpr int SMALL_N = 16 * TILE;  // single-CTA sort up to 32768 keys

template <typename K>
__device__ __forceinline__ unsigned digit_of(K k, int shift) {
    return (unsigned)((k >> shift) & (K)0xff);
}

// Ranks one tile.  wh must be zero on entry; on exit wh[w][d] holds the
// exclusive prefix over warps of digit d's count and tot[d] (if non-null)
// the tile's count of digit d.  Invalid slots get digit 256.  CG: read the
// keys from L2 (data written by other CTAs of the same launch).
template <typename K, bool HV, bool CG = false>
__device__ __forceinline__ void rank_tile(const K *kin, const int *vin, int n, int tile_base,
                                          unsigned (*wh)[256], K *key, int *val, unsigned *dig,
                                          unsigned *rank, int shift) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int base = tile_base + warp * 256;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        int idx = base + r * 32 + lane;
        bool valid = idx < n;
        key[r] = valid ? (CG ? __ldcg(kin + idx) : kin[idx]) : (K)0;
        if (HV) val[r] = valid ? (CG ? __ldcg(vin + idx) : vin[idx]) : 0;
        unsigned d = valid ? digit_of(key[r], shift) : 256u;
        dig[r] = d;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        unsigned lt = peers & ((1u << lane) - 1u);
        unsigned before = d < 256 ? wh[warp][d] : 0u;
        rank[r] = before + __popc(lt);
        __syncwarp();
        if (d < 256 && lt == 0) wh[warp][d] = before + __popc(peers);
        __syncwarp();
    }
}

// tiles of the live input: n, or *d_n (clamped to n) when a device count is
// given.  Returns 0 when the single-CTA kernel sorts the input instead.
__device__ __forceinline__ int live_tiles(int n, const int *d_n) {
    if (d_n) {
        n = min(n, *d_n);
        if (n <= SMALL_N) return 0;
    }
    return (n + TILE - 1) / TILE;
}

// per-tile digit counts, digit-major with rows as long as the live tile
// count (tiles past the live input neither count nor get scanned)
template <typename K>
__global__ void __launch_bounds__(TPB) k_hist(const K *keys, int n, const int *d_n, int shift,
                                              unsigned *hist) {
    HFCR_PDL_WAIT();
    const int nba = live_tiles(n, d_n);
    if ((int)blockIdx.x >= nba) return;
    if (d_n) n = min(n, *d_n);
    __shared__ unsigned h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    int base = blockIdx.x * TILE;
    for (int i = threadIdx.x; i < TILE; i += TPB) {
        int idx = base + i;
        if (idx < n) atomicAdd(&h[digit_of(keys[idx], shift)], 1u);
    }
    __syncthreads();
    hist[threadIdx.x * nba + blockIdx.x] = h[threadIdx.x];
}

// exclusive scan of a[0..m) in place by the calling CTA (NT threads),
// starting from carry; returns carry + the sum to every thread.  CGL: read
// a from L2 (written by other CTAs of the same launch).  Chunks of 4 NT: each thread loads 4
// consecutive elements (coalesced across the warp), the CTA scans the
// per-thread sums, and a running carry links the chunks.
template <int NT, bool CGL = false>
__device__ __forceinline__ unsigned block_scan_excl(unsigned *a, int m, unsigned carry = 0) {
    __shared__ unsigned ws[32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    constexpr int NW = NT / 32;
    for (int base = 0; base < m; base += 4 * NT) {
        const int i0 = base + 4 * t;
        unsigned v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = i0 + q < m ? (CGL ? __ldcg(a + i0 + q) : a[i0 + q]) : 0u;
        const unsigned sum = v[0] + v[1] + v[2] + v[3];
        unsigned x = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) ws[w] = x;
        __syncthreads();
        if (w == 0) {
            unsigned y = lane < NW ? ws[lane] : 0u;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned z = __shfl_up_sync(0xffffffffu, y, o);
                if (lane >= o) y += z;
            }
            if (lane < NW) ws[lane] = y;
        }
        __syncthreads();
        unsigned e = carry + x - sum + (w ? ws[w - 1] : 0u);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (i0 + q < m) a[i0 + q] = e;
            e += v[q];
        }
        carry += ws[NW - 1];
        __syncthreads();  // ws is rewritten by the next chunk
    }
    return carry;
}

// exclusive scan of a[0..m) (m clamped to *d_m) by one CTA; total to *d_total
__global__ void __launch_bounds__(1024) k_scan1(unsigned *a, int m, const int *d_m, int *d_total) {
    HFCR_PDL_WAIT();
    if (d_m) m = min(m, *d_m);
    unsigned total = block_scan_excl<1024>(a, m);
    if (threadIdx.x == 0 && d_total) *d_total = (int)total;
}

// the histogram scan of one pass: CTA d scans digit d's row of tile counts
// in place and writes the digit's total to tot[d]
__global__ void __launch_bounds__(TPB) k_scan_rows(unsigned *hist, int n, const int *d_n,
                                                   unsigned *tot) {
    HFCR_PDL_WAIT();
    const int nba = live_tiles(n, d_n);
    if (!nba) return;
    unsigned total = block_scan_excl<TPB>(hist + blockIdx.x * nba, nba);
    if (threadIdx.x == 0) tot[blockIdx.x] = total;
}

// Multi-CTA exclusive scan of a[0..m) (m clamped to *d_m), for the flag
// scans: CTA b owns chunk b of SCAN_CHUNK elements.  The first kernel
// writes each chunk's sum to part[b]; the second adds up part[0..b) in each
// CTA (at most a few thousand values) and scans its chunk from there.
constexpr int SCAN_CHUNK = 4096;

__global__ void __launch_bounds__(TPB) k_scan_reduce(const unsigned *a, int m, const int *d_m,
                                                     unsigned *part) {
    HFCR_PDL_WAIT();
    __shared__ unsigned ws[TPB / 32];
    if (d_m) m = min(m, *d_m);
    const int base = blockIdx.x * SCAN_CHUNK;
    if (base >= m) return;
    const int end = min(m, base + SCAN_CHUNK);
    unsigned x = 0;
    for (int i = base + threadIdx.x; i < end; i += TPB) x += a[i];
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned tsum = 0;
        for (int w = 0; w < TPB / 32; ++w) tsum += ws[w];
        part[blockIdx.x] = tsum;
    }
}

__global__ void __launch_bounds__(TPB) k_scan_down(unsigned *a, int m, const int *d_m,
                                                   const unsigned *part, int *d_total) {
    HFCR_PDL_WAIT();
    __shared__ unsigned ws[TPB / 32];
    if (d_m) m = min(m, *d_m);
    const int base = blockIdx.x * SCAN_CHUNK;
    const int nlive = (m + SCAN_CHUNK - 1) / SCAN_CHUNK;
    if (m == 0 && blockIdx.x == 0 && threadIdx.x == 0 && d_total) *d_total = 0;
    if (base >= m) return;
    unsigned x = 0;
    for (int i = threadIdx.x; i < (int)blockIdx.x; i += TPB) x += part[i];
#pragma unroll
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = x;
    __syncthreads();
    unsigned off = 0;
    for (int w = 0; w < TPB / 32; ++w) off += ws[w];
    __syncthreads();  // ws is reused by the scan below
    const int len = min(m - base, SCAN_CHUNK);
    unsigned total = block_scan_excl<TPB>(a + base, len, off);
    if ((int)blockIdx.x == nlive - 1 && threadIdx.x == 0 && d_total) *d_total = (int)total;
}

template <typename K, bool HV>
__global__ void __launch_bounds__(TPB) k_scatter(const K *kin, const int *vin, K *kout, int *vout,
                                                 int n, const int *d_n, int shift,
                                                 const unsigned *hist, const unsigned *tot) {
    HFCR_PDL_WAIT();
    const int nba = live_tiles(n, d_n);
    if ((int)blockIdx.x >= nba) return;
    if (d_n) n = min(n, *d_n);
    __shared__ unsigned wh[TPB / 32][256];
    __shared__ unsigned dbase[256];
    __shared__ unsigned wsum[TPB / 32];
    // first output position of each digit: exclusive scan of the digit totals
    {
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        const unsigned c = tot[threadIdx.x];
        unsigned x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            unsigned y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        unsigned before = 0;
        for (int q = 0; q < w; ++q) before += wsum[q];
        dbase[threadIdx.x] = before + x - c;
    }
    for (int i = threadIdx.x; i < (TPB / 32) * 256; i += TPB) (&wh[0][0])[i] = 0;
    __syncthreads();
    K key[ROUNDS];
    int val[ROUNDS];
    unsigned dig[ROUNDS], rank[ROUNDS];
    rank_tile<K, HV>(kin, vin, n, blockIdx.x * TILE, wh, key, val, dig, rank, shift);
    __syncthreads();
    unsigned run = 0;
    for (int w = 0; w < TPB / 32; ++w) {
        unsigned c = wh[w][threadIdx.x];
        wh[w][threadIdx.x] = run;
        run += c;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        unsigned d = dig[r];
        if (d < 256) {
            unsigned pos = dbase[d] + hist[d * nba + blockIdx.x] + wh[warp][d] + rank[r];
            kout[pos] = key[r];
            if (HV) vout[pos] = val[r];
        }
    }
}

// One CTA sorts all passes.  Returns (via *d_flip) nothing: the caller
// knows the pass count and hence the buffer holding the result.
template <typename K, bool HV>
__device__ __forceinline__ void sort_small_body(K *k0, int *v0, K *k1, int *v1, int n, int bits);

template <typename K, bool HV>
__global__ void __launch_bounds__(TPB) k_sort_small(K *k0, int *v0, K *k1, int *v1, int n,
                                                    const int *d_n, int bits) {
    HFCR_PDL_WAIT();
    if (d_n) n = min(n, *d_n);
    if (n > SMALL_N) return;  // the multi-CTA kernels sort it
    sort_small_body<K, HV>(k0, v0, k1, v1, n, bits);
}

// Each segment of a batch (CTA i: the keys of segment i, rows i and i + 1 of
// the segment table, column col) sorted on its own by the single-CTA body,
// in place at its offset, over the low `bits` bits (the higher bits are the
// segment number, constant within a segment).  A segment longer than
// SMALL_N is left alone and *d_rest gets n_total: the caller's global sort
// then sorts everything.
template <typename K, bool HV>
__global__ void __launch_bounds__(TPB) k_sort_segments(K *k0, int *v0, K *k1, int *v1, int n_total,
                                                       const int *segs, int col, int nseg, int bits,
                                                       int *d_rest) {
    HFCR_PDL_WAIT();
    const int i = blockIdx.x;
    if (i >= nseg) return;
    const int a = min(max(segs[4 * i + col], 0), n_total);
    const int b = min(max(segs[4 * (i + 1) + col], a), n_total);
    const int n = b - a;
    if (n > SMALL_N) {
        if (threadIdx.x == 0) *d_rest = n_total;
        return;
    }
    if (n <= 1) {
        // a sort of one key still ends in the buffer the passes would use
        if (n == 1 && threadIdx.x == 0 && (((bits + 7) / 8) & 1)) {
            k1[a] = k0[a];
            if (HV) v1[a] = v0[a];
        }
        return;
    }
    sort_small_body<K, HV>(k0 + a, HV ? v0 + a : v0, k1 + a, HV ? v1 + a : v1, n, bits);
}

template <typename K, bool HV>
__device__ __forceinline__ void sort_small_body(K *k0, int *v0, K *k1, int *v1, int n, int bits) {
    __shared__ unsigned wh[TPB / 32][256];
    __shared__ unsigned off[256];
    __shared__ unsigned cnt[256];
    K *kin = k0, *kout = k1;
    int *vin = v0, *vout = v1;
    for (int shift = 0; shift < bits; shift += 8) {
        // digit totals over the whole input
        cnt[threadIdx.x] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < n; i += TPB) atomicAdd(&cnt[digit_of(kin[i], shift)], 1u);
        __syncthreads();
        if (threadIdx.x < 32) {
            // exclusive scan of 256 counts by one warp (8 per lane)
            const int lane = threadIdx.x;
            unsigned loc[8], s = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) { loc[q] = cnt[lane * 8 + q]; s += loc[q]; }
            unsigned v = s;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            unsigned e = v - s;
#pragma unroll
            for (int q = 0; q < 8; ++q) { off[lane * 8 + q] = e; e += loc[q]; }
        }
        __syncthreads();
        for (int tb = 0; tb < n; tb += TILE) {
            for (int i = threadIdx.x; i < (TPB / 32) * 256; i += TPB) (&wh[0][0])[i] = 0;
            __syncthreads();
            K key[ROUNDS];
            int val[ROUNDS];
            unsigned dig[ROUNDS], rank[ROUNDS];
            rank_tile<K, HV>(kin, vin, n, tb, wh, key, val, dig, rank, shift);
            __syncthreads();
            unsigned run = 0;
            for (int w = 0; w < TPB / 32; ++w) {
                unsigned c = wh[w][threadIdx.x];
                wh[w][threadIdx.x] = run;
                run += c;
            }
            cnt[threadIdx.x] = run;  // tile total of this digit
            __syncthreads();
            const int warp = threadIdx.x >> 5;
#pragma unroll
            for (int r = 0; r < ROUNDS; ++r) {
                unsigned d = dig[r];
                if (d < 256) {
                    unsigned pos = off[d] + wh[warp][d] + rank[r];
                    kout[pos] = key[r];
                    if (HV) vout[pos] = val[r];
                }
            }
            __syncthreads();
            off[threadIdx.x] += cnt[threadIdx.x];
            __syncthreads();
        }
        K *tk = kin; kin = kout; kout = tk;
        int *tv = vin; vin = vout; vout = tv;
        __syncthreads();
    }
}

// Grid-wide barrier of k_sort_coop: a monotone arrival counter (zeroed
// before the launch); barrier number e is passed when it reaches
// e * gridDim.x.  The cooperative launch makes every CTA co-resident; the
// spin is bounded all the same: after ~0.5 s the CTA records ST_TIMEOUT in
// *status and every CTA that sees the flag leaves the kernel (the sort's
// output is then invalid and the caller reports HFCR_ERR_TIMEOUT).
constexpr long long BARRIER_SPIN_LIMIT = 1ll << 22;

__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned epoch, uint32_t *status) {
    __shared__ int failed;
    __syncthreads();
    if (threadIdx.x == 0) {
        failed = 0;
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned target = epoch * gridDim.x;
        long long spins = 0;
        while (true) {
            unsigned seen;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(seen) : "l"(bar) : "memory");
            if (seen >= target) break;
            if (*(volatile uint32_t *)status & ST_TIMEOUT) { failed = 1; break; }
            if (++spins > BARRIER_SPIN_LIMIT) {
                atomicOr(status, ST_TIMEOUT);
                failed = 1;
                break;
            }
            __nanosleep(100);
        }
        __threadfence();
    }
    __syncthreads();
    return failed == 0;
}

// All passes of the multi-CTA sort in one cooperative launch (the per-pass
// kernels below remain the fallback where cooperative launch is refused):
// the grid (at most the co-resident CTAs)
// walks the live tiles in each phase, with grid-wide barriers between the
// histogram, the digit-row scans and the scatter.  When the live count fits
// the single-CTA kernel (a count on the device) every CTA returns at once
// (every CTA reads the same count before any barrier, so none waits alone).  Data written by other
// CTAs in the same launch (keys, histogram rows, digit totals) is read with
// L2 loads (__ldcg), never through a possibly stale L1 line.
template <typename K, bool HV>
__global__ void __launch_bounds__(TPB) k_sort_coop(K *k0, int *v0, K *k1, int *v1, int n,
                                                   const int *d_n, int bits, unsigned *hist,
                                                   unsigned *tot, unsigned *bar, uint32_t *status) {
    HFCR_PDL_WAIT();
    if (d_n) n = min(n, *d_n);
    if (n <= SMALL_N) return;
    unsigned epoch = 0;
    const int nba = (n + TILE - 1) / TILE;
    __shared__ unsigned wh[TPB / 32][256];
    __shared__ unsigned dbase[256];
    __shared__ unsigned wsum[TPB / 32];
    K *kin = k0, *kout = k1;
    int *vin = v0, *vout = v1;
    for (int shift = 0; shift < bits; shift += 8) {
        for (int b = blockIdx.x; b < nba; b += gridDim.x) {
            wh[0][threadIdx.x] = 0;
            __syncthreads();
            const int base = b * TILE;
            for (int i = threadIdx.x; i < TILE; i += TPB) {
                const int idx = base + i;
                if (idx < n) atomicAdd(&wh[0][digit_of(__ldcg(kin + idx), shift)], 1u);
            }
            __syncthreads();
            hist[threadIdx.x * nba + b] = wh[0][threadIdx.x];
            __syncthreads();
        }
        if (!grid_barrier(bar, ++epoch, status)) return;
        for (int d = blockIdx.x; d < 256; d += gridDim.x) {
            const unsigned total = block_scan_excl<TPB, true>(hist + d * nba, nba);
            if (threadIdx.x == 0) tot[d] = total;
        }
        if (!grid_barrier(bar, ++epoch, status)) return;
        {
            const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
            const unsigned c = __ldcg(tot + threadIdx.x);
            unsigned x = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (lane == 31) wsum[w] = x;
            __syncthreads();
            unsigned before = 0;
            for (int q = 0; q < w; ++q) before += wsum[q];
            dbase[threadIdx.x] = before + x - c;
            __syncthreads();
        }
        for (int b = blockIdx.x; b < nba; b += gridDim.x) {
            for (int i = threadIdx.x; i < (TPB / 32) * 256; i += TPB) (&wh[0][0])[i] = 0;
            __syncthreads();
            K key[ROUNDS];
            int val[ROUNDS];
            unsigned dig[ROUNDS], rank[ROUNDS];
            rank_tile<K, HV, true>(kin, vin, n, b * TILE, wh, key, val, dig, rank, shift);
            __syncthreads();
            unsigned run = 0;
            for (int w = 0; w < TPB / 32; ++w) {
                unsigned c = wh[w][threadIdx.x];
                wh[w][threadIdx.x] = run;
                run += c;
            }
            __syncthreads();
            const int warp = threadIdx.x >> 5;
#pragma unroll
            for (int r = 0; r < ROUNDS; ++r) {
                const unsigned d = dig[r];
                if (d < 256) {
                    const unsigned pos = dbase[d] + __ldcg(hist + d * nba + b) + wh[warp][d] + rank[r];
                    kout[pos] = key[r];
                    if (HV) vout[pos] = val[r];
                }
            }
            __syncthreads();
        }
        if (!grid_barrier(bar, ++epoch, status)) return;
        K *tk = kin; kin = kout; kout = tk;
        int *tv = vin; vin = vout; vout = tv;
    }
}

// co-resident CTAs of k_sort_coop<K, HV> on this device (0: cooperative
// launch unavailable)
template <typename K, bool HV>
int coop_grid() {
    static int g[64] = {0};
    static bool done[64] = {false};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!done[dev]) {
        int per_sm = 0, sms = 0, coop = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sort_coop<K, HV>, TPB, 0) ==
                cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) == cudaSuccess && coop)
            g[dev] = per_sm * sms;
        else
            cudaGetLastError();
        done[dev] = true;
    }
    return g[dev];
}

template <typename K, bool HV>
bool radix_sort_impl(K *k0, int *v0, K *k1, int *v1, int n, const int *d_n, int bits,
                     SortTemp &t, cudaStream_t s) {
    // n: the element count (d_n == null) or an upper bound of *d_n
    int passes = (bits + 7) / 8;
    if (n <= 0 || passes == 0) return false;
    if (n <= SMALL_N || d_n) {
        // with a device count the single CTA sorts whenever *d_n <= SMALL_N
        // and the multi-CTA kernels below return at once; otherwise the reverse
        { launch_pdl(k_sort_small<K, HV>, 1, TPB, 0, s, k0, v0, k1, v1, n, d_n,
                     passes * 8); note_launch(); }
        if (n <= SMALL_N) return passes & 1;
    }
    int nb = (n + TILE - 1) / TILE;
    // the digit totals sit in the spare row after the largest histogram
    unsigned *tot = t.hist + 256 * (size_t)(t.max_blocks - 1);
    if (d_n) {  // with a host count the per-pass kernels are as fast and launch no idle work
        int grid = coop_grid<K, HV>();
        if (grid > nb) grid = nb;
        if (grid > 0) {
            int bits8 = passes * 8;
            unsigned *bar = t.hist + 256 * (size_t)(t.max_blocks - 2);
            uint32_t *status = t.status;
            cudaMemsetAsync(bar, 0, sizeof(unsigned), s);
            void *args[] = {&k0, &v0, &k1, &v1, &n, (void *)&d_n, &bits8, &t.hist, &tot, &bar, &status};
            if (status && cudaLaunchCooperativeKernel((const void *)k_sort_coop<K, HV>, grid, TPB, args, 0, s) ==
                cudaSuccess) {
                note_launch();
                return passes & 1;
            }
            cudaGetLastError();
        }
    }
    K *kin = k0, *kout = k1;
    int *vin = v0, *vout = v1;
    for (int p = 0; p < passes; ++p) {
        int shift = 8 * p;
        { launch_pdl(k_hist<K>, nb, TPB, 0, s, kin, n, d_n, shift, t.hist); note_launch(); }
        { launch_pdl(k_scan_rows, 256, TPB, 0, s, t.hist, n, d_n, tot); note_launch(); }
        { launch_pdl(k_scatter<K, HV>, nb, TPB, 0, s, kin, vin, kout, vout, n, d_n, shift, t.hist,
                     tot); note_launch(); }
        K *tk = kin; kin = kout; kout = tk;
        int *tv = vin; vin = vout; vout = tv;
    }
    return passes & 1;
}

}  // namespace

int sort_blocks_for(int n) { return (n + TILE - 1) / TILE; }

bool radix_sort_u64v_segments(unsigned long long *k0, int *v0, unsigned long long *k1, int *v1,
                              int n, int bits, const int *segs, int col, int nseg, int seg_bits,
                              int *d_rest, SortTemp &t, cudaStream_t s) {
    const int passes = (bits + 7) / 8;
    if (n <= 0 || passes == 0) return false;
    // the segment sorts take as many passes as the global sort, or one more
    // (a copy over constant bits) so that both leave the result in one buffer
    int sp = (seg_bits + 7) / 8;
    if ((sp & 1) != (passes & 1)) ++sp;
    cudaMemsetAsync(d_rest, 0, sizeof(int), s);
    { launch_pdl(k_sort_segments<unsigned long long, true>, nseg, TPB, 0, s, k0, v0, k1, v1, n,
                 segs, col, nseg,
                                                                     sp * 8, d_rest); note_launch(); }
    // everything again, globally, only if a segment was too long for one CTA
    return radix_sort_impl<unsigned long long, true>(k0, v0, k1, v1, n, d_rest, bits, t, s);
}

bool radix_sort_u32(unsigned *k0, int *v0, unsigned *k1, int *v1, int n, int bits, SortTemp &t,
                    cudaStream_t s) {
    if (v0) return radix_sort_impl<unsigned, true>(k0, v0, k1, v1, n, nullptr, bits, t, s);
    return radix_sort_impl<unsigned, false>(k0, nullptr, k1, nullptr, n, nullptr, bits, t, s);
}
bool radix_sort_u64(unsigned long long *k0, int *v0, unsigned long long *k1, int *v1, int n,
                    int bits, SortTemp &t, cudaStream_t s) {
    if (v0)
        return radix_sort_impl<unsigned long long, true>(k0, v0, k1, v1, n, nullptr, bits, t, s);
    return radix_sort_impl<unsigned long long, false>(k0, nullptr, k1, nullptr, n, nullptr, bits, t,
                                                      s);
}
bool radix_sort_u64_dev(unsigned long long *k0, unsigned long long *k1, const int *d_n, int cap,
                        int bits, SortTemp &t, cudaStream_t s) {
    return radix_sort_impl<unsigned long long, false>(k0, nullptr, k1, nullptr, cap, d_n, bits, t, s);
}
bool radix_sort_u64v_dev(unsigned long long *k0, int *v0, unsigned long long *k1, int *v1,
                         const int *d_n, int cap, int bits, SortTemp &t, cudaStream_t s) {
    return radix_sort_impl<unsigned long long, true>(k0, v0, k1, v1, cap, d_n, bits, t, s);
}
bool radix_sort_u32_dev(unsigned *k0, int *v0, unsigned *k1, int *v1, const int *d_n, int cap,
                        int bits, SortTemp &t, cudaStream_t s) {
    return radix_sort_impl<unsigned, true>(k0, v0, k1, v1, cap, d_n, bits, t, s);
}

void scan_flags_dev(unsigned *flags, const int *d_n, int cap, int *d_total, SortTemp &t,
                    cudaStream_t s) {
    if (cap <= SCAN_CHUNK) {
        { launch_pdl(k_scan1, 1, 1024, 0, s, flags, cap, d_n, d_total); note_launch(); }
        return;
    }
    const int nc = (cap + SCAN_CHUNK - 1) / SCAN_CHUNK;
    { launch_pdl(k_scan_reduce, nc, TPB, 0, s, flags, cap, d_n, t.hist); note_launch(); }
    { launch_pdl(k_scan_down, nc, TPB, 0, s, flags, cap, d_n, t.hist, d_total); note_launch(); }
}

int bits_for(long long n) {
    int b = 1;
    while ((1ll << b) < n) ++b;
    return b;
}

}  // namespace hfcr
