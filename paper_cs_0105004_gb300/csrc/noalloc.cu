// Ring-road stepping on caller-owned device buffers, without any device
// allocation by the library.
//
// Some callers cannot let a library call cudaMalloc: code that runs inside a
// framework which owns every byte of device memory through its own pool,
// plugins that are handed fixed buffers and must not grow the process's
// footprint, or hosts that pre-plan all memory before a long run.  For them
// ts_ring_step_noalloc advances a periodic circle road (the 1-lane and
// 3-lane circles of Sec. 5) whose state the caller keeps in its own device
// buffers.  It runs the same link kernel as ts_step; what that kernel needs
// besides the caller's buffers (the scenario table, the tile list, the
// control block, the per-step partial statistics and the moving/location
// bitplanes) lives in one file-scope __device__ array, fixed in size, that
// every device which loads this library holds until the process exits.
#include <algorithm>
#include <cuda.h>
#include <mutex>
#include <vector>

#include "internal.h"
#include "transsim.h"

namespace tsim {

namespace {

constexpr uint32_t kNoAllocMaxCells = 1u << 17;  // cells per lane
constexpr uint32_t kNoAllocMaxSteps = 1024;      // steps per call
constexpr uint32_t kNoAllocMaxCols = kNoAllocMaxCells / 32u;
constexpr uint32_t kNoAllocMaxTiles = (kNoAllocMaxCols + kWarpTileCols - 1) / kWarpTileCols;
constexpr uint32_t kNoAllocMaxWords = kNoAllocMaxCols * (uint32_t)kMaxLanes;

// Byte offsets inside the scratch array.
constexpr size_t kOffTable = 0;
constexpr size_t kOffCtrl = 512;
constexpr size_t kOffLink = 768;
constexpr size_t kOffCount = 1024;
constexpr size_t kOffTiles = 1280;
constexpr size_t kOffCols = kOffTiles + ((sizeof(uint2) * kNoAllocMaxTiles + 255u) / 256u) * 256u;
constexpr size_t kOffAux = kOffCols + sizeof(uint4) * kNoAllocMaxCols;
constexpr size_t kOffStats = kOffAux + sizeof(uint4) * kNoAllocMaxCols;
constexpr size_t kOffPlanes = kOffStats + sizeof(StatRec) * kStatsRing;  // mov0, mov1, loc0, loc1
constexpr size_t kScratchBytes = kOffPlanes + 4ull * 4ull * kNoAllocMaxWords;

static_assert(sizeof(ScenDev) <= 512, "table entry fits its slot");
static_assert(sizeof(Ctrl) <= 256, "control block fits its slot");

__device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the scratch array for the context current on each
// device ordinal (looked up once per device and context).
std::mutex g_mu;
struct ScratchAddr {
    CUcontext ctx;
    unsigned char *ptr;
};
std::vector<ScratchAddr> g_scratch;
typedef CUresult (*CtxGetCurrent)(CUcontext *);
CtxGetCurrent g_ctx_get = nullptr;

ts_status bad(ts_status s, const char *msg) {
    set_last_error(msg);
    return s;
}

// Writes this call's scenario entry, control block, link record, tile list
// and column table into the scratch (all of it rewritten by every call) and
// clears the statistics ring.  One ring link of ncols columns and `lanes`
// lanes: tiles of 30 columns (one tile if the ring has at most 30).
__global__ void setup_ring(ScenDev sd, Ctrl ctrl, uint4 link, uint32_t ncols, uint32_t lanes, ScenDev *table,
                           Ctrl *d_ctrl, uint4 *d_link, uint32_t *d_count, uint2 *tiles, uint4 *cols, uint4 *aux,
                           StatRec *stats) {
    const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    const uint32_t n_tiles = (ncols + kWarpTileCols - 1) / kWarpTileCols;  // whole ring if it fits one tile
    if (tid == 0) {
        *table = sd;
        *d_ctrl = ctrl;
        *d_link = link;
        *d_count = n_tiles;
    }
    for (uint32_t j = tid; j < ncols; j += nth) {
        cols[j] = make_uint4(j * lanes, 0u, j | (lanes << 20) | (1u << 23), link.y);
        aux[j] = make_uint4(0u, 0u, 0u, 0u);  // a ring has no link-end buffers and no signal
    }
    for (uint32_t i = tid; i < n_tiles; i += nth) {
        const uint32_t c0 = i * kWarpTileCols;
        const uint32_t n = ncols - c0 < (uint32_t)kWarpTileCols ? ncols - c0 : (uint32_t)kWarpTileCols;
        tiles[i] = make_uint2((n - 1u) << 24, c0);
    }
    unsigned long long *z = reinterpret_cast<unsigned long long *>(stats);
    for (uint32_t i = tid; i < kStatsRing * (uint32_t)(sizeof(StatRec) / 8); i += nth) z[i] = 0ull;
}

// Derives the moving and location bitplanes of the caller's state of step
// `first` (payload in set cur = first & 1) and adds its vehicle count, speed
// sum and digest into the control block.
__global__ void prep_ring(ScenDev D, uint32_t lanes, uint32_t words, uint32_t cur) {
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long act = 0, sv = 0, hs = 0;
    if (w < words) {
        const uint32_t o = D.occ[cur][w];
        uint32_t mv = 0;
        const uint32_t k = w % lanes, x0 = (w / lanes) * 32u;
        for (uint32_t m = o; m; m &= m - 1) {
            const uint32_t i = (uint32_t)__ffs(m) - 1u;
            const uint32_t v = (uint32_t)D.vel[cur][w * 32u + i];
            if (v) mv |= 1u << i;
            sv += v;
            hs += vehicle_term(D.vid[cur][w * 32u + i] & kIdMask, 0u, k, x0 + i, v);
        }
        act = (unsigned long long)__popc(o);
        D.mov[cur][w] = mv;
        D.loc[cur][w] = cur ? o : 0u;  // location bit set = payload in set 1
        D.mov[cur ^ 1u][w] = 0u;
        D.loc[cur ^ 1u][w] = 0u;
    }
    for (int d = 16; d; d >>= 1) {
        act += __shfl_xor_sync(0xffffffffu, act, d);
        sv += __shfl_xor_sync(0xffffffffu, sv, d);
        hs += __shfl_xor_sync(0xffffffffu, hs, d);
    }
    if ((threadIdx.x & 31u) == 0u && act) {
        atomicAdd(&D.ctrl->active, act);
        atomicAdd(&D.ctrl->sum_v, sv);
        atomicAdd(&D.ctrl->hash, hs);
    }
}

// Moves every vehicle's payload of the final state into set f, where the
// caller reads it.
__global__ void finish_ring(ScenDev D, uint32_t words, uint32_t f) {
    const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= words) return;
    const uint32_t o = D.occ[f][w], l = D.loc[f][w];
    const uint32_t away = o & (f ? ~l : l);
    for (uint32_t m = away; m; m &= m - 1) {
        const uint32_t i = (uint32_t)__ffs(m) - 1u;
        D.vel[f][w * 32u + i] = D.vel[f ^ 1u][w * 32u + i];
        D.vid[f][w * 32u + i] = D.vid[f ^ 1u][w * 32u + i];
    }
}

// Per-step statistics from the step records: counts as recorded, running
// values as the values at `first` plus the changes of steps first..t
// (inclusive scan, one block of kNoAllocMaxSteps threads).
__global__ void gather_ring_stats(const StatRec *recs, const Ctrl *ctrl, unsigned long long first, uint32_t n,
                                  ts_stats *out) {
    __shared__ unsigned long long sc[3][kNoAllocMaxSteps];
    const uint32_t i = threadIdx.x;
    const StatRec *r = recs + ((first + i) & (kStatsRing - 1));
    sc[0][i] = i < n ? r->d_active : 0ull;
    sc[1][i] = i < n ? r->d_sum_v : 0ull;
    sc[2][i] = i < n ? r->d_hash : 0ull;
    __syncthreads();
    for (uint32_t d = 1; d < kNoAllocMaxSteps; d <<= 1) {
        unsigned long long a[3];
        for (int f = 0; f < 3; ++f) a[f] = i >= d ? sc[f][i - d] : 0ull;
        __syncthreads();
        for (int f = 0; f < 3; ++f) sc[f][i] += a[f];
        __syncthreads();
    }
    if (i >= n) return;
    ts_stats o;
    o.step = first + i;
    o.active = ctrl->active + sc[0][i];
    o.buffered = 0;
    o.waiting = 0;
    o.arrived = 0;
    o.lane_changes = r->lane_changes;
    o.transfers = 0;
    o.inserted = 0;
    o.sum_v = ctrl->sum_v + sc[1][i];
    o.vehicle_updates = r->vehicle_updates;
    o.state_hash = ctrl->hash + sc[2][i];
    o.moving = r->moving;
    out[i] = o;
}

}  // namespace
}  // namespace tsim

using namespace tsim;

extern "C" {

// Declared in include/transsim.h; see the comment there.
ts_status ts_ring_step_noalloc(uint32_t cells, uint32_t lanes, const ts_params *params, uint64_t first_step,
                               uint32_t n_steps, uint32_t *dev_occ0, uint32_t *dev_occ1, int8_t *dev_vel0,
                               int8_t *dev_vel1, uint32_t *dev_vid0, uint32_t *dev_vid1, ts_stats *dev_stats_out,
                               void *cuda_stream) {
    if (!params) return bad(TS_ERR_INVALID, "null params");
    if (cells < 32 || cells > kNoAllocMaxCells || cells % 32u != 0u)
        return bad(TS_ERR_INVALID, "ring cells must be a multiple of 32 in 32..131072");
    if (lanes < 1 || lanes > (uint32_t)kMaxLanes) return bad(TS_ERR_INVALID, "lanes must be 1..4");
    if (params->vmax < 1 || params->vmax > (uint32_t)kMaxVmax) return bad(TS_ERR_INVALID, "vmax must be 1..15");
    if (n_steps > kNoAllocMaxSteps) return bad(TS_ERR_INVALID, "at most 1024 steps per call");
    if (!dev_occ0 || !dev_occ1 || !dev_vel0 || !dev_vel1 || !dev_vid0 || !dev_vid1 || !dev_stats_out)
        return bad(TS_ERR_INVALID, "null buffer");
    if (n_steps == 0) return TS_OK;
    // an error left pending by earlier work of the caller is reported as
    // such, and not taken for a failure of this call's launches
    const cudaError_t pending = cudaPeekAtLastError();
    if (pending != cudaSuccess) return bad(TS_ERR_CUDA, "a CUDA error was pending before the call");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return bad(TS_ERR_CUDA, "cudaGetDevice failed");
    unsigned char *base = nullptr;
    {
        // once per device and context, with that device current: the
        // host-side name of the array is not a device address, so ask the
        // runtime for it (again after the device's context was replaced, for
        // example by cudaDeviceReset)
        std::lock_guard<std::mutex> lock(g_mu);
        CUcontext ctx = nullptr;
        if (g_ctx_get == nullptr) {
            // the driver's cuCtxGetCurrent through the runtime (the library
            // does not link the driver library itself)
            void *fn = nullptr;
            cudaDriverEntryPointQueryResult q;
            if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
                q == cudaDriverEntryPointSuccess)
                g_ctx_get = reinterpret_cast<CtxGetCurrent>(fn);
        }
        if (g_ctx_get == nullptr || g_ctx_get(&ctx) != CUDA_SUCCESS) ctx = nullptr;
        if ((size_t)dev >= g_scratch.size()) g_scratch.resize((size_t)dev + 1, ScratchAddr{nullptr, nullptr});
        ScratchAddr &sa = g_scratch[dev];
        if (!sa.ptr || ctx == nullptr || sa.ctx != ctx) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p)
                return bad(TS_ERR_CUDA, "cudaGetSymbolAddress failed");
            sa.ptr = static_cast<unsigned char *>(p);
            sa.ctx = ctx;
        }
        base = sa.ptr;
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    ScenDev *d_table = reinterpret_cast<ScenDev *>(base + kOffTable);
    Ctrl *d_ctrl = reinterpret_cast<Ctrl *>(base + kOffCtrl);
    uint4 *d_link = reinterpret_cast<uint4 *>(base + kOffLink);
    uint2 *d_tiles = reinterpret_cast<uint2 *>(base + kOffTiles);
    uint4 *d_cols = reinterpret_cast<uint4 *>(base + kOffCols);
    uint4 *d_aux = reinterpret_cast<uint4 *>(base + kOffAux);
    uint32_t *d_count = reinterpret_cast<uint32_t *>(base + kOffCount);
    StatRec *d_stats = reinterpret_cast<StatRec *>(base + kOffStats);
    uint32_t *d_planes = reinterpret_cast<uint32_t *>(base + kOffPlanes);

    const uint32_t ncols = cells / 32u, words = ncols * lanes;
    const uint32_t n_tiles = (ncols + kWarpTileCols - 1) / kWarpTileCols;
    ScenDev sd{};
    sd.lk_info = d_link;
    sd.col_info = d_cols;
    sd.col_aux = d_aux;
    sd.n_cols = ncols;
    sd.occ[0] = dev_occ0;
    sd.occ[1] = dev_occ1;
    sd.mov[0] = d_planes;
    sd.mov[1] = d_planes + kNoAllocMaxWords;
    sd.loc[0] = d_planes + 2u * kNoAllocMaxWords;
    sd.loc[1] = d_planes + 3u * kNoAllocMaxWords;
    sd.vel[0] = dev_vel0;
    sd.vel[1] = dev_vel1;
    sd.vid[0] = dev_vid0;
    sd.vid[1] = dev_vid1;
    sd.ctrl = d_ctrl;
    sd.stats = d_stats;
    sd.n_sub = 1;
    sd.vmax = params->vmax;
    sd.p_threshold = params->p_threshold;
    sd.seed_lo = (uint32_t)(params->seed & 0xFFFFFFFFull);
    sd.seed_hi = (uint32_t)(params->seed >> 32);
    sd.lane_change = params->lane_change ? 1u : 0u;
    sd.n_links = 1;
    Ctrl ctrl{};
    ctrl.base = first_step;
    ctrl.target = first_step + n_steps;
    const uint4 link = make_uint4(0u, cells, lanes | (1u << 8), 0u);
    // the scratch keeps the previous call's contents: the set-up kernel
    // rewrites all of it that this call reads (its arguments travel by value,
    // no host buffer is involved) and clears the statistics it accumulates
    // into; every launch is checked as it is made
    const uint32_t cur = (uint32_t)(first_step & 1ull), fin = (uint32_t)((first_step + n_steps) & 1ull);
    setup_ring<<<32, 256, 0, s>>>(sd, ctrl, link, ncols, lanes, d_table, d_ctrl, d_link, d_count, d_tiles, d_cols,
                                  d_aux, d_stats);
    if (cudaGetLastError() != cudaSuccess) return bad(TS_ERR_CUDA, "set-up kernel launch failed");
    prep_ring<<<(words + 255u) / 256u, 256, 0, s>>>(sd, lanes, words, cur);
    if (cudaGetLastError() != cudaSuccess) return bad(TS_ERR_CUDA, "kernel launch failed");
    const int want = (int)((n_tiles + kLinkWarpsPerBlock - 1) / kLinkWarpsPerBlock);
    const int grid = std::max(1, std::min<int>(want, max_link_blocks(false)));
    for (uint32_t i = 0; i < n_steps; ++i) {
        launch_link_kernel(d_table, d_tiles, d_count, i, grid, s, false, false, false);
        if (cudaGetLastError() != cudaSuccess) return bad(TS_ERR_CUDA, "step kernel launch failed");
    }
    finish_ring<<<(words + 255u) / 256u, 256, 0, s>>>(sd, words, fin);
    if (cudaGetLastError() != cudaSuccess) return bad(TS_ERR_CUDA, "kernel launch failed");
    gather_ring_stats<<<1, kNoAllocMaxSteps, 0, s>>>(d_stats, d_ctrl, first_step, n_steps, dev_stats_out);
    if (cudaGetLastError() != cudaSuccess) return bad(TS_ERR_CUDA, "kernel launch failed");
    return TS_OK;
}

}  // extern "C"
