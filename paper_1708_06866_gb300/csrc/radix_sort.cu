// radix_sort.cu — stable LSD radix sort of uint64 keys (optionally carrying
// uint32 values) and the block-total scan used by the stream compactions.
//
// One histogram pass counts the 8-bit digits of every pass at once; each
// digit pass is then a single read-and-scatter kernel ("onesweep"): a block
// ranks its tile of keys by digit with warp ballots/popc, publishes its digit
// counts, and learns the counts of all earlier tiles by a decoupled
// look-back over a status array.  Every look-back wait is bounded in time;
// a wait that runs out sets DEV_ERR_TIMEOUT and the block skips its writes.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <string>
#include <utility>

#include "tc_internal.cuh"

namespace tc {
namespace {

constexpr int RS_BLOCK = 256;                 // threads per block (== RADIX)
constexpr int RS_ITEMS = 16;                  // keys per thread
#ifndef TC_RS_MIN_BLOCKS
#define TC_RS_MIN_BLOCKS 3                    // resident onesweep blocks per SM (register cap)
#endif
constexpr int RS_TILE = RS_BLOCK * RS_ITEMS;  // keys per tile
constexpr int RS_WARPS = RS_BLOCK / 32;
constexpr int RADIX = 256;
constexpr int MAX_PASSES = 8;

// Status word of (tile, digit): [63:60] pass tag (pass + 1), [59:58] kind
// (1 = this tile's count, 2 = inclusive prefix through this tile),
// [57:0] count.  A word whose tag differs from the running pass is "not
// published yet", so one memset per sort serves every pass.  A word carries
// its whole message, so it is written and polled with relaxed accesses (no
// fence).
constexpr uint64_t ST_COUNT_MASK = (1ull << 58) - 1;
__device__ __forceinline__ uint64_t st_word(int pass, uint64_t kind, uint64_t cnt) {
    return ((uint64_t)(pass + 1) << 60) | (kind << 58) | cnt;
}

// Digit mask of pass p for keys of key_bits bits: the last pass of a
// key_bits that is not a multiple of 8 keeps only the bits below key_bits,
// so higher bits never take part in the ordering.
__host__ __device__ __forceinline__ uint32_t digit_mask(int p, int key_bits) {
    const int rem = key_bits - 8 * p;
    return rem >= 8 ? 255u : (1u << rem) - 1u;
}

__global__ void __launch_bounds__(RS_BLOCK) k_histogram(const uint64_t* __restrict__ keys,
                                                        int64_t n, int passes, int key_bits,
                                                        unsigned long long* __restrict__ hist) {
    __shared__ uint32_t sh[MAX_PASSES * RADIX];
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x) sh[i] = 0;
    __syncthreads();
    // HU keys per thread per step, all loaded before the first count
    constexpr int HU = 8;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * HU;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x * HU + threadIdx.x; b < n; b += stride) {
        uint64_t k[HU];
#pragma unroll
        for (int u = 0; u < HU; ++u) {
            const int64_t i = b + (int64_t)u * blockDim.x;
            k[u] = i < n ? keys[i] : 0ull;
        }
#pragma unroll
        for (int u = 0; u < HU; ++u)
            if (b + (int64_t)u * blockDim.x < n)
                for (int p = 0; p < passes; ++p)
                    atomicAdd(&sh[p * RADIX + ((k[u] >> (8 * p)) & digit_mask(p, key_bits))], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * RADIX; i += blockDim.x)
        if (sh[i]) atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

// Per pass (one block each, a thread per digit): exclusive scan of the digit
// counts.
__global__ void __launch_bounds__(RADIX) k_bin_start(unsigned long long* hist) {
    __shared__ unsigned long long sh[RADIX];
    unsigned long long* h = hist + blockIdx.x * RADIX;
    const int d = threadIdx.x;
    sh[d] = h[d];
    __syncthreads();
    // Hillis-Steele inclusive scan in shared memory
    for (int off = 1; off < RADIX; off <<= 1) {
        const unsigned long long add = d >= off ? sh[d - off] : 0ull;
        __syncthreads();
        sh[d] += add;
        __syncthreads();
    }
    h[d] = d == 0 ? 0ull : sh[d - 1];
}

template <bool HAS_VAL>
__global__ void __launch_bounds__(RS_BLOCK, TC_RS_MIN_BLOCKS) k_onesweep(
    const uint64_t* __restrict__ kin, uint64_t* __restrict__ kout,
    const uint32_t* __restrict__ vin, uint32_t* __restrict__ vout, int64_t n, int pass, uint32_t dmask,
    const unsigned long long* __restrict__ bin_start, uint64_t* __restrict__ status,
    unsigned int* __restrict__ tile_counter, int* __restrict__ err, int64_t spin_ns) {
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* s_keys = reinterpret_cast<uint64_t*>(smem);
    uint32_t* s_vals = reinterpret_cast<uint32_t*>(s_keys + RS_TILE);
    // per-warp digit counts, then each (warp, digit)'s first position in the
    // digit-sorted tile
    __shared__ uint32_t s_whist[RS_WARPS * RADIX];
    // per digit: output position of tile position p is s_gofs[d] + p
    __shared__ unsigned long long s_gofs[RADIX];
    __shared__ uint32_t s_scan[33];
    __shared__ int64_t s_tile;
    __shared__ int s_bad;

    const int shift = 8 * pass;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        s_tile = (int64_t)atomicAdd(tile_counter, 1u);
        s_bad = 0;
    }
    for (int i = threadIdx.x; i < RS_WARPS * RADIX; i += RS_BLOCK) s_whist[i] = 0;
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t wbase = tile * RS_TILE + (int64_t)warp * (32 * RS_ITEMS);

    // 1. load the warp's keys (all loads in flight before any ranking),
    // then rank every key among the keys of its warp with the same digit
    uint64_t k[RS_ITEMS];
    uint32_t v[RS_ITEMS];
    uint32_t r[RS_ITEMS];
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const int64_t idx = wbase + i * 32 + lane;
        const bool ok = idx < n;
        k[i] = ok ? kin[idx] : 0ull;
        if (HAS_VAL) v[i] = ok ? vin[idx] : 0u;
    }
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const bool ok = wbase + i * 32 + lane < n;
        const uint32_t d = ok ? (uint32_t)((k[i] >> shift) & dmask) : 256u;
        // lanes with the same digit: one ballot per bit of the 9-bit value
        // (256 marks a lane past the end; ballots measured faster than
        // match.any here)
        unsigned peers = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            const bool bit = (d >> b) & 1u;
            const unsigned bb = __ballot_sync(0xffffffffu, bit);
            peers &= bit ? bb : ~bb;
        }
        const int leader = __ffs(peers) - 1;
        uint32_t b = 0;
        if (lane == leader && d < 256u) {
            b = s_whist[warp * RADIX + d];
            s_whist[warp * RADIX + d] = b + __popc(peers);
        }
        b = __shfl_sync(0xffffffffu, b, leader);
        r[i] = b + __popc(peers & lanemask_lt());
        __syncwarp();
    }
    __syncthreads();

    // 2. per digit: offsets of the warps, tile count, publish, look back
    const int t = threadIdx.x;  // digit owned by this thread
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) {
        const uint32_t c = s_whist[w * RADIX + t];
        s_whist[w * RADIX + t] = tot;
        tot += c;
    }
    uint64_t* my_status = status + tile * RADIX + t;
    st_relaxed_u64(my_status, st_word(pass, tile == 0 ? 2 : 1, tot));
    uint32_t tile_total;
    const uint32_t dstart = block_exclusive_scan(tot, s_scan, &tile_total);
#pragma unroll
    for (int w = 0; w < RS_WARPS; ++w) s_whist[w * RADIX + t] += dstart;

    uint64_t prefix = 0;
    if (tile > 0) {
        int64_t j = tile - 1;
        uint64_t t0 = 0;
        bool bad = false;
        for (;;) {
            const uint64_t st = ld_relaxed_u64(status + j * RADIX + t);
            if ((st >> 60) != (uint64_t)(pass + 1)) {
                const uint64_t now = global_timer_ns();
                if (t0 == 0) t0 = now;
                else if ((int64_t)(now - t0) > spin_ns) { bad = true; break; }
                continue;
            }
            prefix += st & ST_COUNT_MASK;
            if (((st >> 58) & 3) == 2) break;
            if (--j < 0) { bad = true; break; }
        }
        if (bad) {
            atomicOr(err, DEV_ERR_TIMEOUT);
            s_bad = 1;
        }
        st_relaxed_u64(my_status, st_word(pass, 2, prefix + tot));
    }
    s_gofs[t] = bin_start[t] + prefix - dstart;  // modulo 2^64: adding p >= dstart is exact
    __syncthreads();

    // 3. place keys in digit order within the tile, then write runs out
#pragma unroll
    for (int i = 0; i < RS_ITEMS; ++i) {
        const int64_t idx = wbase + i * 32 + lane;
        if (idx < n) {
            const uint32_t d = (uint32_t)((k[i] >> shift) & dmask);
            const uint32_t p = s_whist[warp * RADIX + d] + r[i];
            s_keys[p] = k[i];
            if (HAS_VAL) s_vals[p] = v[i];
        }
    }
    __syncthreads();
    if (s_bad) return;
    const int64_t rem = n - tile * RS_TILE;
    const int tile_n = rem < RS_TILE ? (int)rem : RS_TILE;
    for (int p = threadIdx.x; p < tile_n; p += RS_BLOCK) {
        const uint64_t key = s_keys[p];
        const uint32_t d = (uint32_t)((key >> shift) & dmask);
        const unsigned long long pos = s_gofs[d] + (unsigned long long)p;
        if (pos < (unsigned long long)n) {
            kout[pos] = key;
            if (HAS_VAL) vout[pos] = s_vals[p];
        } else {
            atomicOr(err, DEV_ERR_BOUNDS);
        }
    }
}

constexpr size_t dyn_smem(bool has_val) {
    return (size_t)RS_TILE * 8 + (has_val ? (size_t)RS_TILE * 4 : 0);
}

// One block: exclusive scan of `count` uint32 values in place; the grand
// total goes to *grand.
__global__ void __launch_bounds__(1024) k_scan_totals(uint32_t* v, int64_t count,
                                                      uint64_t* grand) {
    __shared__ uint32_t s_scan[33];
    __shared__ unsigned long long s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < count; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const uint32_t x = i < count ? v[i] : 0u;
        uint32_t tot;
        const uint32_t ex = block_exclusive_scan(x, s_scan, &tot);
        if (i < count) v[i] = (uint32_t)(s_carry + ex);
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand = s_carry;
}

}  // namespace

int radix_sort_u64(uint64_t* keys, uint64_t* keys_alt, uint32_t* vals, uint32_t* vals_alt,
                   int64_t n, int key_bits, int* dev_err, cudaStream_t s) {
    if (n <= 1) return TC_OK;
    const int passes = (key_bits + 7) / 8;
    if (passes < 1 || passes > MAX_PASSES) return fail(TC_EINVAL, "radix_sort_u64: key_bits");
    const int64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    if (tiles > 0x7fffffffLL) return fail(TC_EOVERFLOW, "radix_sort_u64: too many keys");
    Scratch sc(s);
    unsigned long long* hist;
    uint64_t* status;
    unsigned int* counters;
    TC_TRY(sc.alloc(&hist, (int64_t)passes * RADIX));
    TC_TRY(sc.alloc(&status, tiles * RADIX));
    TC_TRY(sc.alloc(&counters, MAX_PASSES));
    TC_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * passes * RADIX, s));
    TC_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(uint64_t) * tiles * RADIX, s));
    TC_CUDA_TRY(cudaMemsetAsync(counters, 0, sizeof(unsigned int) * MAX_PASSES, s));

    const int hblocks = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * 4);
    k_histogram<<<hblocks, RS_BLOCK, 0, s>>>(keys, n, passes, key_bits, hist);
    TC_LAUNCH_CHECK("k_histogram");
    k_bin_start<<<passes, RADIX, 0, s>>>(hist);
    TC_LAUNCH_CHECK("k_bin_start");

    const bool has_val = vals != nullptr;
    // process-wide function attributes: set once per device (constant values)
    static std::atomic<unsigned long long> attr_done{0};
    int dev = 0;
    TC_CUDA_TRY(cudaGetDevice(&dev));
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_done.load() & bit)) {
        TC_CUDA_TRY(cudaFuncSetAttribute(k_onesweep<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn_smem(true)));
        TC_CUDA_TRY(cudaFuncSetAttribute(k_onesweep<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn_smem(false)));
        attr_done.fetch_or(bit);
    }
    const int64_t spin = spin_limit_ns();
    uint64_t *ka = keys, *kb = keys_alt;
    uint32_t *va = vals, *vb = vals_alt;
    for (int p = 0; p < passes; ++p) {
        if (has_val)
            k_onesweep<true><<<(unsigned)tiles, RS_BLOCK, dyn_smem(true), s>>>(
                ka, kb, va, vb, n, p, digit_mask(p, key_bits), hist + p * RADIX, status,
                counters + p, dev_err, spin);
        else
            k_onesweep<false><<<(unsigned)tiles, RS_BLOCK, dyn_smem(false), s>>>(
                ka, kb, nullptr, nullptr, n, p, digit_mask(p, key_bits), hist + p * RADIX,
                status, counters + p, dev_err, spin);
        TC_LAUNCH_CHECK("k_onesweep");
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (ka != keys) {  // odd number of passes: result sits in the alt buffers
        TC_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        if (has_val)
            TC_CUDA_TRY(
                cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    return TC_OK;
}

// ---------------------------------------------------------------------------
// Sorting without allocation.  tc_sort_keys_static is for callers that cannot
// allocate device memory at the point of the call: code whose memory is
// entirely owned by another allocator (a framework's caching pool holding
// the free memory), code running where an allocation would break a
// pre-planned memory budget or a real-time deadline, and code that must not
// touch the device allocator at all.  Its scratch lives in one file-scope
// device array of fixed size, shared by every call in the process.
namespace {

constexpr int64_t kStaticSortMaxKeys = int64_t(1) << 20;  // TC_SORT_STATIC_MAX_KEYS
constexpr int64_t kStaticTiles = kStaticSortMaxKeys / RS_TILE;
constexpr size_t kAltBytes = sizeof(uint64_t) * kStaticSortMaxKeys;
constexpr size_t kStatusBytes = sizeof(uint64_t) * kStaticTiles * RADIX;
constexpr size_t kHistBytes = sizeof(unsigned long long) * MAX_PASSES * RADIX;
constexpr size_t kCtlBytes = 256;  // pass counters, then the error word
constexpr size_t kStaticSortBytes = kAltBytes + kStatusBytes + kHistBytes + kCtlBytes;

static_assert(kStaticSortMaxKeys == TC_SORT_STATIC_MAX_KEYS, "header limit");
static_assert(kStaticSortBytes == TC_SORT_STATIC_SCRATCH_BYTES, "header scratch size");

// Alt key buffer | tile status words | digit histograms | counters + error.
static __device__ __align__(256) unsigned char g_sort_scratch[kStaticSortBytes];

std::mutex g_static_mu;
void* g_static_ptr[64] = {nullptr};  // device address of g_sort_scratch, per device

// Once per device, with that device current: the array's device address (in
// host code its name is only a host-side stand-in) and the kernels' shared
// memory attribute.
int static_sort_setup(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (dev < 0 || dev >= 64) return fail(TC_EINVAL, "tc_sort_keys_static: device index");
    if (!g_static_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(TC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        }
        TC_CUDA_TRY(cudaFuncSetAttribute(k_onesweep<false>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)dyn_smem(false)));
        g_static_ptr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_static_ptr[dev]);
    return TC_OK;
}

}  // namespace

}  // namespace tc

extern "C" int tc_sort_keys_static(uint64_t* keys, int64_t n, int32_t key_bits,
                                   void* cuda_stream) {
    using namespace tc;
    if (n < 0) return fail(TC_EINVAL, "tc_sort_keys_static: n < 0");
    if (n > kStaticSortMaxKeys)
        return fail(TC_EOVERFLOW, "tc_sort_keys_static: n exceeds TC_SORT_STATIC_MAX_KEYS (2^20); "
                                  "use the allocating entry points for larger inputs");
    if (key_bits < 1 || key_bits > 64) return fail(TC_EINVAL, "tc_sort_keys_static: key_bits");
    if (n > 0 && !keys) return fail(TC_EINVAL, "tc_sort_keys_static: keys is NULL");
    if (n > 0 && is_host_pointer(keys))
        return fail(TC_EINVAL, "tc_sort_keys_static: keys must be device memory");
    int dev = 0;
    TC_CUDA_TRY(cudaGetDevice(&dev));
    unsigned char* base = nullptr;
    TC_TRY(static_sort_setup(dev, &base));
    if (n <= 1) return TC_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    uint64_t* alt = reinterpret_cast<uint64_t*>(base);
    uint64_t* status = reinterpret_cast<uint64_t*>(base + kAltBytes);
    unsigned long long* hist =
        reinterpret_cast<unsigned long long*>(base + kAltBytes + kStatusBytes);
    unsigned int* counters =
        reinterpret_cast<unsigned int*>(base + kAltBytes + kStatusBytes + kHistBytes);
    int* err = reinterpret_cast<int*>(counters + MAX_PASSES);
    const int passes = (key_bits + 7) / 8;
    const int64_t tiles = (n + RS_TILE - 1) / RS_TILE;
    // the array keeps the previous call's contents: clear what must start at zero
    TC_CUDA_TRY(cudaMemsetAsync(hist, 0, sizeof(unsigned long long) * passes * RADIX, s));
    TC_CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(uint64_t) * tiles * RADIX, s));
    TC_CUDA_TRY(cudaMemsetAsync(counters, 0, kCtlBytes, s));
    const int hblocks = (int)std::min<int64_t>(tiles, (int64_t)num_sms() * 4);
    k_histogram<<<hblocks, RS_BLOCK, 0, s>>>(keys, n, passes, key_bits, hist);
    TC_LAUNCH_CHECK("k_histogram");
    k_bin_start<<<passes, RADIX, 0, s>>>(hist);
    TC_LAUNCH_CHECK("k_bin_start");
    const int64_t spin = spin_limit_ns();
    uint64_t *ka = keys, *kb = alt;
    for (int p = 0; p < passes; ++p) {
        k_onesweep<false><<<(unsigned)tiles, RS_BLOCK, dyn_smem(false), s>>>(
            ka, kb, nullptr, nullptr, n, p, digit_mask(p, key_bits), hist + p * RADIX, status,
            counters + p, err, spin);
        TC_LAUNCH_CHECK("k_onesweep");
        std::swap(ka, kb);
    }
    if (ka != keys)
        TC_CUDA_TRY(cudaMemcpyAsync(keys, ka, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    int h = 0;
    TC_CUDA_TRY(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, s));
    TC_CUDA_TRY(cudaStreamSynchronize(s));
    if (h & DEV_ERR_TIMEOUT) return fail(TC_ETIMEDOUT, "tc_sort_keys_static: a wait ran out of time");
    if (h) return fail(TC_ECUDA, "tc_sort_keys_static: internal bounds check failed");
    return TC_OK;
}

namespace tc {

int scan_block_totals(uint32_t* totals, int64_t count, uint64_t* grand_total_dev,
                      cudaStream_t s) {
    k_scan_totals<<<1, 1024, 0, s>>>(totals, count, grand_total_dev);
    TC_LAUNCH_CHECK("k_scan_totals");
    return TC_OK;
}

}  // namespace tc
