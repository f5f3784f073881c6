// Device building blocks of the stable LSD radix sort (8-bit digits), the
// CTA-wide exclusive scan and the bounded grid-wide barrier, shared by the
// sort kernels (sort.cu) and the fused response-setup kernel (solve.cu).
//
// Tile = 256 threads x 8 rounds of 32 keys = 2048 keys.  Within a tile each
// warp owns 256 consecutive keys and ranks them round by round: lanes with
// the same digit are found with __match_any_sync, a lane's rank is the
// number of equal-digit lanes before it plus the warp's running count of
// that digit (kept in shared memory), which preserves input order.  Per-
// warp counts are then prefix-summed across the 8 warps, and a tile's
// global offset for a digit comes from the digit-major scan of all tiles'
// histograms.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace hfcr {

namespace {

constexpr int TPB = 256;
constexpr int ROUNDS = 8;
constexpr int TILE = TPB * ROUNDS;  // 2048
constexpr int SMALL_N = 16 * TILE;  // single-CTA sort up to 32768 keys
constexpr int HIST_BATCH = 8;       // keys a thread loads at once for a digit count
constexpr int FEW_TILES = 16;       // grid sorts of at most this many tiles skip the scan phase

// shared memory of one sorting CTA (the kernel declares it once, so that a
// kernel holding several sorts, or a sort and other phases, can overlay it)
struct SortSmem {
    unsigned wh[TPB / 32][256];
    unsigned off[256];
    unsigned cnt[256];
    unsigned wsum[TPB / 32];
};

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
    // every load of the tile first (independent, in flight together), then
    // the rounds of ranking
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int idx = base + r * 32 + lane;
        const bool valid = idx < n;
        key[r] = valid ? (CG ? __ldcg(kin + idx) : kin[idx]) : (K)0;
        if (HV) val[r] = valid ? (CG ? __ldcg(vin + idx) : vin[idx]) : 0;
    }
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const bool valid = base + r * 32 + lane < n;
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

// One CTA (TPB threads) sorts all passes, walking its tiles in order.  The
// result is in (k1, v1) after an odd number of passes, else in (k0, v0).
// CG: every key and value is read from L2 (inputs written by other CTAs of
// the same launch).
template <typename K, bool HV, bool CG = false>
__device__ __forceinline__ void sort_small_body(K *k0, int *v0, K *k1, int *v1, int n, int bits,
                                                SortSmem &sm) {
    unsigned (*wh)[256] = sm.wh;
    unsigned *off = sm.off, *cnt = sm.cnt;
    K *kin = k0, *kout = k1;
    int *vin = v0, *vout = v1;
    for (int shift = 0; shift < bits; shift += 8) {
        // digit totals over the whole input
        cnt[threadIdx.x] = 0;
        __syncthreads();
        for (int i0 = 0; i0 < n; i0 += HIST_BATCH * TPB) {
            unsigned dg[HIST_BATCH];
#pragma unroll
            for (int q = 0; q < HIST_BATCH; ++q) {  // loads first, in flight together
                const int i = i0 + q * TPB + threadIdx.x;
                dg[q] = i < n ? digit_of(CG ? __ldcg(kin + i) : kin[i], shift) : 256u;
            }
#pragma unroll
            for (int q = 0; q < HIST_BATCH; ++q)
                if (dg[q] < 256u) atomicAdd(&cnt[dg[q]], 1u);
        }
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
            rank_tile<K, HV, CG>(kin, vin, n, tb, wh, key, val, dig, rank, shift);
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

// Grid-wide barrier: a monotone arrival counter (zeroed before the launch);
// barrier number e is passed when it reaches e * parts, parts = the CTAs
// taking part (gridDim.x unless given; CTAs beyond it must not call).  The
// cooperative launch makes every CTA co-resident; the spin is bounded all
// the same: after ~0.5 s the CTA records ST_TIMEOUT in *status and every
// CTA that sees the flag leaves the kernel (its output is then invalid and
// the caller reports HFCR_ERR_TIMEOUT).
constexpr long long BARRIER_SPIN_LIMIT = 1ll << 22;

__device__ __forceinline__ bool grid_barrier(unsigned *bar, unsigned epoch, uint32_t *status,
                                             unsigned parts = 0) {
    __shared__ int failed;
    __syncthreads();
    if (threadIdx.x == 0) {
        failed = 0;
        __threadfence();
        atomicAdd(bar, 1u);
        const unsigned target = epoch * (parts ? parts : gridDim.x);
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

// All passes of the multi-CTA sort by every CTA of a cooperative launch:
// the grid walks the tiles in each phase, with grid-wide barriers between
// the histogram, the digit-row scans and the scatter (with at most
// FEW_TILES tiles and a CTA per tile, each CTA derives its offsets itself
// and the scan phase and its barrier drop out).  hist holds 256 rows
// of ceil(n / TILE) tile counts, tot 256 digit totals.  Data written by
// other CTAs (keys, histogram rows, digit totals) is read with L2 loads
// (__ldcg), never through a possibly stale L1 line.  parts: the CTAs taking
// part (the first ones; all when 0).  Returns false when a barrier gave up;
// the result is in (k1, v1) after an odd number of passes.
template <typename K, bool HV>
__device__ __forceinline__ bool sort_grid_body(K *k0, int *v0, K *k1, int *v1, int n, int bits,
                                               unsigned *hist, unsigned *tot, unsigned *bar,
                                               unsigned &epoch, uint32_t *status, SortSmem &sm,
                                               unsigned parts = 0) {
    const int nba = (n + TILE - 1) / TILE;
    const int P = parts ? (int)parts : (int)gridDim.x;  // CTAs taking part (the first P)
    unsigned (*wh)[256] = sm.wh;
    unsigned *dbase = sm.off, *wsum = sm.wsum;
    K *kin = k0, *kout = k1;
    int *vin = v0, *vout = v1;
    for (int shift = 0; shift < bits; shift += 8) {
        for (int b = blockIdx.x; b < nba; b += P) {
            wh[0][threadIdx.x] = 0;
            __syncthreads();
            const int base = b * TILE;
            unsigned dg[ROUNDS];
#pragma unroll
            for (int q = 0; q < ROUNDS; ++q) {  // loads first, in flight together
                const int idx = base + q * TPB + threadIdx.x;
                dg[q] = idx < n ? digit_of(__ldcg(kin + idx), shift) : 256u;
            }
#pragma unroll
            for (int q = 0; q < ROUNDS; ++q)
                if (dg[q] < 256u) atomicAdd(&wh[0][dg[q]], 1u);
            __syncthreads();
            hist[threadIdx.x * nba + b] = wh[0][threadIdx.x];
            __syncthreads();
        }
        if (!grid_barrier(bar, ++epoch, status, P)) return false;
        if (nba <= P && nba <= FEW_TILES) {
            // one tile per CTA: each CTA with a tile derives its digit offsets
            // itself (thread d: digit d's count over all tiles and over the
            // tiles before its own), so the pass needs no scan phase
            const int b = blockIdx.x;
            if (b < nba) {
                const int d = threadIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
                unsigned total = 0, before = 0;
                for (int q = 0; q < nba; ++q) {
                    const unsigned c = __ldcg(hist + d * nba + q);
                    total += c;
                    if (q < b) before += c;
                }
                unsigned x = total;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    unsigned y = __shfl_up_sync(0xffffffffu, x, o);
                    if (lane >= o) x += y;
                }
                if (lane == 31) wsum[w] = x;
                __syncthreads();
                unsigned pre = 0;
                for (int q = 0; q < w; ++q) pre += wsum[q];
                dbase[d] = pre + x - total + before;
                for (int i = threadIdx.x; i < (TPB / 32) * 256; i += TPB) (&wh[0][0])[i] = 0;
                __syncthreads();
                K key[ROUNDS];
                int val[ROUNDS];
                unsigned dig[ROUNDS], rank[ROUNDS];
                rank_tile<K, HV, true>(kin, vin, n, b * TILE, wh, key, val, dig, rank, shift);
                __syncthreads();
                unsigned run = 0;
                for (int q = 0; q < TPB / 32; ++q) {
                    unsigned c = wh[q][threadIdx.x];
                    wh[q][threadIdx.x] = run;
                    run += c;
                }
                __syncthreads();
#pragma unroll
                for (int r = 0; r < ROUNDS; ++r) {
                    const unsigned dg = dig[r];
                    if (dg < 256) {
                        const unsigned pos = dbase[dg] + wh[w][dg] + rank[r];
                        kout[pos] = key[r];
                        if (HV) vout[pos] = val[r];
                    }
                }
            }
            if (!grid_barrier(bar, ++epoch, status, P)) return false;
            K *tk = kin; kin = kout; kout = tk;
            int *tv = vin; vin = vout; vout = tv;
            continue;
        }
        for (int d = blockIdx.x; d < 256; d += P) {
            const unsigned total = block_scan_excl<TPB, true>(hist + d * nba, nba);
            if (threadIdx.x == 0) tot[d] = total;
        }
        if (!grid_barrier(bar, ++epoch, status, P)) return false;
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
        for (int b = blockIdx.x; b < nba; b += P) {
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
        if (!grid_barrier(bar, ++epoch, status, P)) return false;
        K *tk = kin; kin = kout; kout = tk;
        int *tv = vin; vin = vout; vout = tv;
    }
    return true;
}

}  // namespace

}  // namespace hfcr
