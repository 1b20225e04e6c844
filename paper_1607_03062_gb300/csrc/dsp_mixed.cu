// dsp_mixed.cu -- the FP32_MIXED evolve kernel on contiguous tiles of 1024
// points (every scheme and grid shape).  Shared device code is in
// dsp_device.cuh.

#include "dsp_device.cuh"

namespace dsp {
namespace {

// The launch's steps on the tile's packs one at a time (G = 1): the series
// level's degrees (DC, DS) are compile-time constants.
template <int SCHEME, int DC, int DS>
__device__ __forceinline__ bool run_level(const ReqDesc &R, unsigned char *smem, uint64_t *bars,
                                          int *err, MixedPack (&pk)[kMixedSpt / 2])
{
    constexpr int NP = kMixedSpt / 2;
    if constexpr (SCHEME == 2) {
        const auto single = [&](const float4 &e) {
#pragma unroll
            for (int k = 0; k < NP; ++k)
                step_magnus2<DC, DS>(pk[k], e);
        };
        return run_steps<float4>(R, smem, bars, err, single);
    } else {
        return run_steps<float2>(R, smem, bars, err, [&](const float2 &e) {
#pragma unroll
            for (int k = 0; k < NP; ++k) {
                if constexpr (SCHEME == 0)
                    step_exact2<DC, DS>(pk[k], e);
                else
                    step_strang<DC, DS>(pk[k], e);
            }
        });
    }
}

template <int SCHEME, int L>
__device__ __forceinline__ bool dispatch_level(const ReqDesc &R, unsigned char *smem,
                                               uint64_t *bars, int *err,
                                               MixedPack (&pk)[kMixedSpt / 2])
{
    if constexpr (L + 1 < kNumLevels) {
        if (R.level != L)
            return dispatch_level<SCHEME, L + 1>(R, smem, bars, err, pk);
    }
    return run_level<SCHEME, kLevelsF32[L].dc, kLevelsF32[L].ds>(R, smem, bars, err, pk);
}

// Tan-normalised groups of G steps (every scheme), tan series of degree DT.
template <int SCHEME, int G, int DT>
__device__ __forceinline__ bool run_tan(const ReqDesc &R, unsigned char *smem, uint64_t *bars,
                                        int *err, MixedPack (&pk)[kMixedSpt / 2])
{
    constexpr int NP = kMixedSpt / 2;
    if constexpr (SCHEME == 2) {
        return run_step_groups<float4, G>(
            R, smem, bars, err,
            [&](const float4 &e) {
#pragma unroll
                for (int k = 0; k < NP; ++k)
                    step_single_tan_magnus<G, DT>(pk[k], e);
            },
            [&](const float4 *e) {
#pragma unroll
                for (int k = 0; k < NP; ++k)
                    step_group_tan_magnus<G, DT>(pk[k], e);
            });
    } else {
        return run_step_groups<float2, G>(
            R, smem, bars, err,
            [&](const float2 &e) {
#pragma unroll
                for (int k = 0; k < NP; ++k)
                    step_single_tan<G, DT, SCHEME>(pk[k], e);
            },
            [&](const float2 *e) {
#pragma unroll
                for (int k = 0; k < NP; ++k)
                    step_group_tan<G, DT, SCHEME>(pk[k], e);
            });
    }
}

template <int SCHEME, int G, int I>
__device__ __forceinline__ bool dispatch_tan_degree(const ReqDesc &R, unsigned char *smem,
                                                    uint64_t *bars, int *err,
                                                    MixedPack (&pk)[kMixedSpt / 2])
{
    constexpr int DT = kTanDegrees[I];
    if constexpr (I + 1 < kNumTanDegrees) {
        if (R.tdeg != DT)
            return dispatch_tan_degree<SCHEME, G, I + 1>(R, smem, bars, err, pk);
    }
    return run_tan<SCHEME, G, DT>(R, smem, bars, err, pk);
}

template <int SCHEME>
__device__ __forceinline__ bool run_mixed(const ReqDesc &R, unsigned char *smem, uint64_t *bars,
                                          int *err, MixedPack (&pk)[kMixedSpt / 2])
{
    if (R.group == kGroupMax)
        return dispatch_tan_degree<SCHEME, kGroupMax, 0>(R, smem, bars, err, pk);
    if (R.group == 8)
        return dispatch_tan_degree<SCHEME, 8, 0>(R, smem, bars, err, pk);
    if (R.group == 4)
        return dispatch_tan_degree<SCHEME, 4, 0>(R, smem, bars, err, pk);
    if (R.group == 2)
        return dispatch_tan_degree<SCHEME, 2, 0>(R, smem, bars, err, pk);
    return dispatch_level<SCHEME, 0>(R, smem, bars, err, pk);
}

template <int SCHEME>
__device__ void body_mixed(const ReqDesc &R, int tile, unsigned char *smem, uint64_t *bars,
                           int *err)
{
    constexpr int S = kMixedSpt;
    const int tid = threadIdx.x;
    const int64_t base = static_cast<int64_t>(tile) * kTilePoints;
    const double vs = R.valley > 0 ? 1.0 : -1.0;
    float4 *hi_plane = static_cast<float4 *>(R.state);
    float4 *lo_plane = hi_plane + R.n_points;

    MixedPoint pt[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t idx = base + s * kMixedThreads + tid;
        const bool valid = idx < R.n_points;
        double px = 0.0, py = 0.0;
        if (valid) {
            px = grid_node(R.px_min, R.hx, idx % R.nx);
            py = grid_node(R.py_min, R.hy, R.row0 + idx / R.nx);
        }
        // valley K- is stepped as K+ on -P: the table holds -dt*A, here -dt*p
        const double tx = vs * (R.dt * px), ty = vs * (R.dt * py);
        pt[s].pxh = static_cast<float>(tx);
        pt[s].pxl = static_cast<float>(tx - static_cast<double>(pt[s].pxh));
        pt[s].pyh = static_cast<float>(ty);
        pt[s].pyl = static_cast<float>(ty - static_cast<double>(pt[s].pyh));
        if (R.fresh || !valid) {
            double ar = 1.0, ai = 0.0, br = 0.0, bi = 0.0;  // identity column
            if (!R.init_identity)
                initial_spinor(px + R.a_in[0], py + R.a_in[1], vs, ar, ai, br, bi);
            pt[s].ar = static_cast<float>(ar);
            pt[s].lar = static_cast<float>(ar - static_cast<double>(pt[s].ar));
            pt[s].ai = static_cast<float>(ai);
            pt[s].lai = static_cast<float>(ai - static_cast<double>(pt[s].ai));
            pt[s].br = static_cast<float>(br);
            pt[s].lbr = static_cast<float>(br - static_cast<double>(pt[s].br));
            pt[s].bi = static_cast<float>(bi);
            pt[s].lbi = static_cast<float>(bi - static_cast<double>(pt[s].bi));
        } else {
            const float4 h = hi_plane[idx], l = lo_plane[idx];
            pt[s].ar = h.x; pt[s].ai = h.y; pt[s].br = h.z; pt[s].bi = h.w;
            pt[s].lar = l.x; pt[s].lai = l.y; pt[s].lbr = l.z; pt[s].lbi = l.w;
        }
    }

    MixedPack pk[S / 2];  // FP32x2: spinors (2k, 2k + 1) share each instruction
#pragma unroll
    for (int k = 0; k < S / 2; ++k)
        pk[k] = pack_points(pt[2 * k], pt[2 * k + 1]);
    const bool ok = run_mixed<SCHEME>(R, smem, bars, err, pk);
#pragma unroll
    for (int k = 0; k < S / 2; ++k)
        unpack_points(pk[k], pt[2 * k], pt[2 * k + 1]);
    if (!ok)
        return;

    // the table stages are free now: they hold the density slots
    float2 *red = reinterpret_cast<float2 *>(smem);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t idx = base + s * kMixedThreads + tid;
        float2 c = make_float2(0.0f, 0.0f);
        if (idx < R.n_points) {
            if (R.store_state) {
                hi_plane[idx] = make_float4(pt[s].ar, pt[s].ai, pt[s].br, pt[s].bi);
                lo_plane[idx] = make_float4(pt[s].lar, pt[s].lai, pt[s].lbr, pt[s].lbi);
            }
            if (R.project) {
                const SpinorDF v{pt[s].ar, pt[s].lar, pt[s].ai, pt[s].lai,
                                 pt[s].br, pt[s].lbr, pt[s].bi, pt[s].lbi};
                c = store_point<1>(R.map, idx, project_node<1>(R, idx % R.nx, idx / R.nx, v));
            }
        }
        if (R.project)
            red[s * kMixedThreads + tid] = c;
    }
    if (R.project)
        granule_sums(red, kTilePoints / kGranule, R.partials, (R.n_points + kGranule - 1) / kGranule,
                     [&](int g) { return base / kGranule + g; });
}

// ---------------------------------------------------------------------------
// Kernel
// ---------------------------------------------------------------------------

__global__ void __launch_bounds__(kMixedThreads, kMixedMinBlocks)
    evolve_mixed_kernel(const __grid_constant__ EvolveArgs args)
{
    __shared__ __align__(128) unsigned char smem[2 * kStageBytes];
    __shared__ __align__(8) uint64_t bars[2];
    if (threadIdx.x == 0) {
        mbar_init(&bars[0], 1);
        mbar_init(&bars[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    const int r = find_request(args);
    const ReqDesc &R = args.r[r];
    const int tile = static_cast<int>(blockIdx.x) - R.tile_begin;
    if (!tile_ok(R, tile, R.err))
        return;
    if (R.scheme == 0)
        body_mixed<0>(R, tile, smem, bars, R.err);
    else if (R.scheme == 1)
        body_mixed<1>(R, tile, smem, bars, R.err);
    else
        body_mixed<2>(R, tile, smem, bars, R.err);
}

}  // namespace

cudaError_t launch_evolve_mixed(const EvolveArgs &args, cudaStream_t stream)
{
    if (args.nreq <= 0 || args.total_tiles <= 0)
        return cudaSuccess;
    evolve_mixed_kernel<<<args.total_tiles, kMixedThreads, 0, stream>>>(args);
    return cudaGetLastError();
}

}  // namespace dsp
