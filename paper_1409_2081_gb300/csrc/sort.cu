// Stable LSD radix sort (8-bit digits) and exclusive scans; the tile
// ranking, the CTA scan, the single-CTA and grid-wide sort bodies and the
// grid barrier are in sortdev.cuh.  Inputs of up to SMALL_N keys are
// sorted by one CTA that walks its tiles in order (one launch for all
// passes).  A sort whose count only the device knows launches that CTA and
// one cooperative kernel that runs every multi-CTA pass when the count is
// larger; the segments of a batch can be sorted one CTA each.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"
#include "sortdev.cuh"

namespace hfcr {

namespace {

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
    const int base = blockIdx.x * TILE;
    unsigned dg[ROUNDS];
#pragma unroll
    for (int q = 0; q < ROUNDS; ++q) {  // loads first, in flight together
        const int idx = base + q * TPB + threadIdx.x;
        dg[q] = idx < n ? digit_of(keys[idx], shift) : 256u;
    }
#pragma unroll
    for (int q = 0; q < ROUNDS; ++q)
        if (dg[q] < 256u) atomicAdd(&h[dg[q]], 1u);
    __syncthreads();
    hist[threadIdx.x * nba + blockIdx.x] = h[threadIdx.x];
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

template <typename K, bool HV>
__global__ void __launch_bounds__(TPB) k_sort_small(K *k0, int *v0, K *k1, int *v1, int n,
                                                    const int *d_n, int bits) {
    HFCR_PDL_WAIT();
    if (d_n) n = min(n, *d_n);
    if (n > SMALL_N) return;  // the multi-CTA kernels sort it
    __shared__ SortSmem sm;
    sort_small_body<K, HV>(k0, v0, k1, v1, n, bits, sm);
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
    __shared__ SortSmem sm;
    sort_small_body<K, HV>(k0 + a, HV ? v0 + a : v0, k1 + a, HV ? v1 + a : v1, n, bits, sm);
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
    __shared__ SortSmem sm;
    sort_grid_body<K, HV>(k0, v0, k1, v1, n, bits, hist, tot, bar, epoch, status, sm);
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
