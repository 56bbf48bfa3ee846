// Device-wide exclusive scan of uint64 values with decoupled look-back.
#include "lookback.cuh"

namespace pv {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanThreads * kScanPer;

// workspace: [u32 ticket, pad to 16][u64 states[ntiles]]
size_t scan_ws_bytes(int n) {
    const int tiles = div_up(n < 1 ? 1 : n, kScanTile);
    return 16 + 8 * (size_t)tiles;
}

__global__ void zero_bytes_kernel(uint8_t *p, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = 0;
}

__global__ void __launch_bounds__(kScanThreads) scan_kernel(const uint64_t *__restrict__ in, int n,
                                                            uint64_t *__restrict__ out, uint8_t *ws,
                                                            int32_t *status, uint64_t limit_ns) {
    __shared__ int s_tile;
    __shared__ uint64_t s_warp[kScanThreads / 32];
    __shared__ uint64_t s_excl;
    __shared__ int s_to;
    uint32_t *ticket = reinterpret_cast<uint32_t *>(ws);
    uint64_t *states = reinterpret_cast<uint64_t *>(ws + 16);
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    if (t == 0) { s_tile = (int)atomicAdd(ticket, 1u); s_to = 0; }
    __syncthreads();
    const int tile = s_tile;
    const long long base = (long long)tile * kScanTile + (long long)t * kScanPer;
    uint64_t v[kScanPer], sum = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        sum += v[k];
    }
    // block-level inclusive scan of per-thread sums
    uint64_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint64_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < kScanThreads / 32) s_warp[lane] = w;
    }
    __syncthreads();
    const uint64_t warp_excl = warp ? s_warp[warp - 1] : 0;
    const uint64_t total = s_warp[kScanThreads / 32 - 1];
    if (t == 0) {
        int to = 0;
        s_excl = lookback_exclusive(states, tile, total, &to, limit_ns);
        s_to = to;
    }
    __syncthreads();
    uint64_t run = s_excl + warp_excl + (x - sum);
#pragma unroll
    for (int k = 0; k < kScanPer; k++) {
        run += v[k];
        if (base + k < n) out[base + k + 1] = run;
    }
    if (tile == 0 && t == 0) out[0] = 0;
    if (t == 0 && s_to && status) *status = PIVCO_ERR_TIMEOUT;
}

cudaError_t launch_zero_bytes(uint8_t *p, size_t n, cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    zero_bytes_kernel<<<min(1024, div_up((long long)n, 256)), 256, 0, st>>>(p, n);
    count_launches(1);
    return cudaGetLastError();
}

cudaError_t launch_scan(const uint64_t *in, int n, uint64_t *out, void *ws, int32_t *status, cudaStream_t st) {
    const int tiles = div_up(n < 1 ? 1 : n, kScanTile);
    const size_t wsb = scan_ws_bytes(n);
    zero_bytes_kernel<<<min(256, div_up((long long)wsb, 256)), 256, 0, st>>>(reinterpret_cast<uint8_t *>(ws), wsb);
    count_launches(1);
    scan_kernel<<<tiles, kScanThreads, 0, st>>>(in, n, out, reinterpret_cast<uint8_t *>(ws), status, wait_limit_ns());
    count_launches(1);
    return cudaGetLastError();
}

}  // namespace pv
