// dsp_strip.cu -- the FP32_MIXED evolve kernel on row strips (every scheme,
// grids whose nx is a multiple of 256).  Shared device code is in
// dsp_device.cuh.
//
// Compiled once per scheme and strip height, with -DDSP_STRIP_SCHEME=<0|1|2>
// (EXACT, STRANG_XY, MAGNUS4) and -DDSP_STRIP_NP=<2|1> (packs per thread: 4-row
// or 2-row strips), so that the objects build in parallel; each defines its own
// kernel, launch_evolve_strip_s<SCHEME>_np<NP> and strip_ctas_per_sm_s<SCHEME>_np<NP>.

#include <type_traits>

#include "dsp_device.cuh"

namespace dsp {
namespace {

// ---------------------------------------------------------------------------
// FP32_MIXED on row strips (grids whose nx is a multiple of 256)
//
// A CTA owns kStripRows = 4 rows x kStripThreads = 256 columns; thread t holds
// column c0 + t of each of the 4 rows, as 2 packs (rows 0, 1 and rows 2, 3).
// (A launch's last strips may be 2 rows high, one pack per thread: see
// ReqDesc::strip_h.)  A
// thread's spinors share p_x and the CTA's threads share the 4 p_y, so the part
// of a step's coefficients that depends on dt P_y alone is computed once per row
// and step into a table in shared memory (built for each chunk of steps), and
// the part that depends on dt P_x alone once per thread and step, as scalars.
// Steps taken one at a time (G = 1):
//   EXACT:     rows dt P_y and fl(dt P_y^2); column dt P_x;
//   STRANG_XY: rows cos(dt P_y) - 1 and sin(dt P_y); column cos(dt P_x) - 1 and
//              sin(dt P_x) (with dt P_x = 2a of the split);
//   MAGNUS4:   rows dt Pbar_y and -fl(dt Pbar_y D_x); column dt Pbar_x (and the
//              step's D_y, the same for every thread).
// Tan-normalised groups (G >= 2):
//   EXACT:     rows dt P_y and fl(dt P_y^2); column dt P_x (tan degree 1: rows
//              dt P_y and fl(fl(c1 dt P_y) dt P_y), column dt P_x and fl(c1 dt P_x));
//   STRANG_XY: rows tan(dt P_y); column tan(dt P_x) and sec(dt P_x) - 1;
//   MAGNUS4:   as for its single steps.
// Every operation on a point is the contiguous path's (same operands, same
// order, same rounding), so each point's result is bitwise the same on either
// tiling; only the work per step shrinks.  Coefficient lane-ops per spinor-step
// of the groups: EXACT 3.5 + DT instead of 8 + DT (DT = 1: 3.75 instead of 10);
// STRANG_XY 1 per spinor plus (4 + 2 DT)/4 per thread instead of 9 + 3 DT;
// MAGNUS4 7.5 + DT instead of 12 + DT.
// ---------------------------------------------------------------------------

#if !defined(DSP_STRIP_SCHEME) || !defined(DSP_STRIP_NP)
#error "compile with -DDSP_STRIP_SCHEME=<0|1|2> -DDSP_STRIP_NP=<1|2>"
#endif

// Unroll factors of the strip path: the loop over a launch's groups, and the
// chain inside a group.  4-row strips (measured on the 2048^2 x 1e5-step LZS
// solves, mean ms per solve: x1/x8 272.3, x2/x8 266.8, x1/x16 267.6, x2/x16
// 264.5, x1/x4 280.3); 2-row strips run only in a launch's last wave and keep
// a smaller body.
#ifndef DSP_STRIP_GROUP_UNROLL
#define DSP_STRIP_GROUP_UNROLL (DSP_STRIP_NP == 2 ? 2 : 1)
#endif
#ifndef DSP_STRIP_CHAIN_UNROLL
#define DSP_STRIP_CHAIN_UNROLL (DSP_STRIP_NP == 2 ? 16 : 8)
#endif
constexpr int kStripGroupUnroll = DSP_STRIP_GROUP_UNROLL;
constexpr int kStripChainUnroll = DSP_STRIP_CHAIN_UNROLL;
constexpr int kStripThreads = 256;
constexpr int kStripRows = 4;
constexpr int kStripStage = 4096;             // bytes per staged table chunk
constexpr int kStripChunk = kStripStage / 8;  // most steps per chunk (float2 entries)

// Table entries: float2 (dt A_x, dt A_y) per step; MAGNUS4 float4 (dt Abar_x,
// dt Abar_y, D_x, D_y).
template <int SCHEME>
using StripEntry = typename std::conditional<SCHEME == 2, float4, float2>::type;
static_assert(kStripThreads * kStripRows == kTilePoints, "a strip tile holds kTilePoints points");
static_assert(kStripThreads == kGranule, "a strip row is one density granule");
static_assert(kStripThreads == kStripWidth && kStripRows == kStripHeight, "the host's tiling");

struct StripSmem {
    unsigned char stage[2][kStripStage];  // bulk-copied table entries (StripEntry)
    float4 rows[kStripChunk][2];          // per step, per pack (rows 0, 1 and 2, 3): strip_row
    float ax[kStripChunk];                // per step: dt A_x (MAGNUS4: dt Abar_x)
    float dy[kStripChunk];                // per step, MAGNUS4: D_y
};
static_assert(sizeof(StripSmem) <= 48 * 1024, "static shared memory of one CTA");

// The row part of a step for the two rows of a pack, from dt P_y of each (and,
// for MAGNUS4, the step's D_x), for steps taken one at a time (G = 1):
//   EXACT     {P_y(r0), P_y(r1), fl(P_y(r0)^2), fl(P_y(r1)^2)}
//   STRANG_XY {cy(r0), cy(r1), sb(r0), sb(r1)}, cy = cos b - 1, sb = sin b, b = dt P_y
//   MAGNUS4   {P_y(r0), P_y(r1), -fl(P_y(r0) D_x), -fl(P_y(r1) D_x)}
// each as coeffs_strang / step_magnus2 form it for one lane.
template <int SCHEME, int DC, int DS>
__device__ __forceinline__ float4 strip_row(float y0, float y1, float dx)
{
    if constexpr (SCHEME == 0) {
        return make_float4(y0, y1, __fmul_rn(y0, y0), __fmul_rn(y1, y1));
    } else if constexpr (SCHEME == 2) {
        return make_float4(y0, y1, -__fmul_rn(y0, dx), -__fmul_rn(y1, dx));
    } else {
        const float x0 = vmul(y0, y0), x1 = vmul(y1, y1);
        const float c0 = vmul(vhorner<float, DC, 1, 0>(x0), x0);
        const float c1 = vmul(vhorner<float, DC, 1, 0>(x1), x1);
        const float s0 = vfma(vmul(vhorner<float, DS, 1, 1>(x0), x0), y0, y0);
        const float s1 = vfma(vmul(vhorner<float, DS, 1, 1>(x1), x1), y1, y1);
        return make_float4(c0, c1, s0, s1);
    }
}

// The row part of a step of the tan-normalised groups (coeffs_tan's operations):
//   EXACT     {P_y(r0), P_y(r1), fl(P_y(r0)^2), fl(P_y(r1)^2)}; with tan degree 1
//             {P_y(r0), P_y(r1), fl(fl(c1 P_y(r0)) P_y(r0)), fl(fl(c1 P_y(r1)) P_y(r1))}
//   STRANG_XY {tan b(r0), tan b(r1), 0, 0}, b = dt P_y
//   MAGNUS4   {P_y(r0), P_y(r1), -fl(P_y(r0) D_x), -fl(P_y(r1) D_x)} (coeffs_tan_magnus's)
template <int SCHEME, int DT>
__device__ __forceinline__ float4 strip_row_tan(float y0, float y1, float dx)
{
    if constexpr (SCHEME == 2) {  // coeffs_tan_magnus's row part, as for single steps
        return make_float4(y0, y1, -__fmul_rn(y0, dx), -__fmul_rn(y1, dx));
    } else if constexpr (SCHEME == 0 && DT == 1) {  // coeffs_tan's row part fl(fl(c1 P_y) P_y)
        return make_float4(y0, y1, __fmul_rn(__fmul_rn(kTanC1, y0), y0),
                           __fmul_rn(__fmul_rn(kTanC1, y1), y1));
    } else if constexpr (SCHEME == 0) {
        return make_float4(y0, y1, __fmul_rn(y0, y0), __fmul_rn(y1, y1));
    } else {
        const float x0 = vmul(y0, y0), x1 = vmul(y1, y1);
        const float t0 = vfma(vmul(vseries<float, TanCoef, DT, 1>(x0), x0), y0, y0);
        const float t1 = vfma(vmul(vseries<float, TanCoef, DT, 1>(x1), x1), y1, y1);
        return make_float4(t0, t1, 0.0f, 0.0f);
    }
}

// The column part of a step, from dt P_x = dt p_hi + (dt A_x + dt p_lo):
//   EXACT     a = (P_x, P_x);
//   STRANG_XY a = (cx, cx), b = (sa, sa): cx = cos 2a - 1, sa = sin 2a, 2a = dt P_x;
//   MAGNUS4   a = (P_x, P_x), b = (D_y, D_y) (P_x from dt Abar_x);
// of the tan-normalised groups (strip_col_tan):
//   EXACT     a = (P_x, P_x) (tan degree 1: b = (fl(c1 P_x), fl(c1 P_x)));
//   STRANG_XY a = (tan 2a, tan 2a), b = (sec 2a - 1, sec 2a - 1);
//   MAGNUS4   as for its single steps.
struct StripCol {
    float2 a, b;
};

template <int SCHEME, int DC, int DS>
__device__ __forceinline__ StripCol strip_col(float pxh, float pxl, float ax, float dy)
{
    const float px = __fadd_rn(pxh, __fadd_rn(ax, pxl));
    if constexpr (SCHEME == 0) {
        return StripCol{make_float2(px, px), make_float2(0.0f, 0.0f)};
    } else if constexpr (SCHEME == 2) {
        return StripCol{make_float2(px, px), make_float2(dy, dy)};
    } else {
        const float xx = vmul(px, px);
        const float cx = vmul(vhorner<float, DC, 1, 0>(xx), xx);
        const float sa = vfma(vmul(vhorner<float, DS, 1, 1>(xx), xx), px, px);
        return StripCol{make_float2(cx, cx), make_float2(sa, sa)};
    }
}

template <int SCHEME, int DT>
__device__ __forceinline__ StripCol strip_col_tan(float pxh, float pxl, float ax, float dy)
{
    const float px = __fadd_rn(pxh, __fadd_rn(ax, pxl));
    if constexpr (SCHEME == 2) {
        return StripCol{make_float2(px, px), make_float2(dy, dy)};
    } else if constexpr (SCHEME == 0 && DT == 1) {  // coeffs_tan's column part fl(c1 P_x)
        const float cpx = __fmul_rn(kTanC1, px);
        return StripCol{make_float2(px, px), make_float2(cpx, cpx)};
    } else if constexpr (SCHEME == 0) {
        return StripCol{make_float2(px, px), make_float2(0.0f, 0.0f)};
    } else {
        const float xx = vmul(px, px);
        const float t = vfma(vmul(vseries<float, TanCoef, DT, 1>(xx), xx), px, px);
        const float sc = vmul(vseries<float, SecCoef, DT, 1>(xx), xx);
        return StripCol{make_float2(t, t), make_float2(sc, sc)};
    }
}

// tau of a step for a pack in coeffs_tan's form.
template <int SCHEME, int DT>
__device__ __forceinline__ void strip_coeffs_tan(const StripCol &c, float4 r, float2 &tr,
                                                 float2 &ti)
{
    if constexpr (SCHEME == 0 && DT == 1) {
        const float2 Py = make_float2(r.x, r.y), rY = make_float2(r.z, r.w);
        const float2 t1 = vfma(c.b, c.a, rY);  // c1 theta^2 = tan(theta)/theta - 1
        tr = vfma(t1, Py, Py);
        ti = vfma(t1, c.a, c.a);
    } else if constexpr (SCHEME == 0) {
        const float2 Py = make_float2(r.x, r.y), Py2 = make_float2(r.z, r.w);
        const float2 x = vfma(c.a, c.a, Py2);
        const float2 t1 = vmul(vseries<float2, TanCoef, DT, 1>(x), x);  // tan(theta)/theta - 1
        tr = vfma(t1, Py, Py);
        ti = vfma(t1, c.a, c.a);
    } else {
        const float2 tb = make_float2(r.x, r.y);
        tr = vfma(tb, c.b, tb);
        ti = c.a;
    }
}

// (m, q) of a STRANG_XY step alone for a pack, in coeffs_strang's form.
template <int DC, int DS>
__device__ __forceinline__ void strip_coeffs_strang(const StripCol &c, float4 r, float2 &m,
                                                    float2 &qr, float2 &qi)
{
    const float2 cy = make_float2(r.x, r.y);
    qr = make_float2(r.z, r.w);
    qi = vfma(cy, c.b, c.b);
    m = vfma(c.a, cy, vadd(c.a, cy));
}

// (tau, tz) of a MAGNUS4 step for a pack in coeffs_tan_magnus's form.
template <int DT>
__device__ __forceinline__ void strip_coeffs_tan_magnus(const StripCol &c, float4 r, float2 &tr,
                                                        float2 &ti, float2 &tz)
{
    const float2 Py = make_float2(r.x, r.y), nyx = make_float2(r.z, r.w);
    const float2 nz = vfma(c.a, c.b, nyx);
    const float2 x = vfma(c.a, c.a, vfma(Py, Py, vmul(nz, nz)));
    const float2 t1 = vmul(vseries<float2, TanCoef, DT, 1>(x), x);  // tan|n|/|n| - 1
    tr = vfma(t1, Py, Py);
    ti = vfma(t1, c.a, c.a);
    tz = vfma(t1, nz, nz);
}

// (m, q) of an EXACT step alone, in coeffs_exact2's form.
template <int DC, int DS>
__device__ __forceinline__ void strip_coeffs_exact(const StripCol &c, float4 r, float2 &m,
                                                   float2 &qr, float2 &qi)
{
    const float2 Py = make_float2(r.x, r.y), Py2 = make_float2(r.z, r.w);
    const float2 x = fma2(c.a, c.a, Py2);
    m = mul2(horner2<DC, 1, 0>(x), x);
    const float2 sn = horner2<DS, 0, 1>(x);
    qr = mul2(sn, Py);
    qi = mul2(sn, c.a);
}

template <int SCHEME, int NP>
struct StripThread {
    float pxh, pxl;  // dt p_x of the column, hi + lo
    const StripSmem *sm;

    template <int DC, int DS>
    __device__ __forceinline__ StripCol col(int j) const
    {
        return strip_col<SCHEME, DC, DS>(pxh, pxl, sm->ax[j], SCHEME == 2 ? sm->dy[j] : 0.0f);
    }
    template <int DT>
    __device__ __forceinline__ StripCol col_tan(int j) const
    {
        return strip_col_tan<SCHEME, DT>(pxh, pxl, sm->ax[j], SCHEME == 2 ? sm->dy[j] : 0.0f);
    }
    // the first and a further step of a pack's tan-normalised chain (MAGNUS4 with its
    // sigma_z part, first_z / next_z)
    template <int DT>
    __device__ __forceinline__ void chain_first(TanChain<float2> &ch, const StripCol &c,
                                                float4 r) const
    {
        float2 tr, ti;
        if constexpr (SCHEME == 2) {
            float2 tz;
            strip_coeffs_tan_magnus<DT>(c, r, tr, ti, tz);
            ch.first_z(tr, ti, tz);
        } else {
            strip_coeffs_tan<SCHEME, DT>(c, r, tr, ti);
            ch.first(tr, ti);
        }
    }
    template <int DT>
    __device__ __forceinline__ void chain_next(TanChain<float2> &ch, const StripCol &c,
                                               float4 r) const
    {
        float2 tr, ti;
        if constexpr (SCHEME == 2) {
            float2 tz;
            strip_coeffs_tan_magnus<DT>(c, r, tr, ti, tz);
            ch.next_z(tr, ti, tz);
        } else {
            strip_coeffs_tan<SCHEME, DT>(c, r, tr, ti);
            ch.next(tr, ti);
        }
    }
    // one step alone: step_exact2 (EXACT), step_strang (STRANG_XY), step_magnus2 (MAGNUS4)
    template <int DC, int DS>
    __device__ __forceinline__ void single(MixedPack (&pk)[NP], int j) const
    {
        const StripCol c = col<DC, DS>(j);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            float2 m, qr, qi;
            if constexpr (SCHEME == 0) {
                strip_coeffs_exact<DC, DS>(c, sm->rows[j][q], m, qr, qi);
                apply_exact2(pk[q], m, qr, qi);
            } else if constexpr (SCHEME == 2) {  // step_magnus2's operations
                const float4 r = sm->rows[j][q];
                const float2 Py = make_float2(r.x, r.y), nyx = make_float2(r.z, r.w);
                const float2 nz = fma2(c.a, c.b, nyx);
                const float2 x = fma2(c.a, c.a, fma2(Py, Py, mul2(nz, nz)));
                m = mul2(horner2<DC, 1, 0>(x), x);
                const float2 sn = horner2<DS, 0, 1>(x);
                apply2(pk[q], m, neg2(mul2(sn, nz)), mul2(sn, Py), mul2(sn, c.a));
            } else {
                strip_coeffs_strang<DC, DS>(c, sm->rows[j][q], m, qr, qi);
                apply_group(pk[q], m, bc2(0.0f), qr, qi);
            }
        }
    }
    // a step of a tan-normalised run outside whole groups (step_single_tan,
    // step_single_tan_magnus)
    template <int G, int DT>
    __device__ __forceinline__ void single_tan(MixedPack (&pk)[NP], int j) const
    {
        const StripCol c = col_tan<DT>(j);
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            TanChain<float2> ch;
            chain_first<DT>(ch, c, sm->rows[j][q]);
            ch.template finish<kTanNormDegree(G)>(pk[q]);
        }
    }
    // step_group_tan's (step_group_tan_magnus's) chain, the packs advanced step by step
    template <int G, int DT>
    __device__ __forceinline__ void group_tan(MixedPack (&pk)[NP], int j) const
    {
        TanChain<float2> ch[NP];
        StripCol c = col_tan<DT>(j);
#pragma unroll
        for (int q = 0; q < NP; ++q)
            chain_first<DT>(ch[q], c, sm->rows[j][q]);
        int k = 1;
        if constexpr (SCHEME != 2) {  // the second step, alpha = 1 still
            c = col_tan<DT>(j + 1);
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                float2 tr, ti;
                strip_coeffs_tan<SCHEME, DT>(c, sm->rows[j + 1][q], tr, ti);
                ch[q].second(tr, ti);
            }
            k = 2;
        }
#pragma unroll kStripChainUnroll
        for (; k < G; ++k) {
            c = col_tan<DT>(j + k);
#pragma unroll
            for (int q = 0; q < NP; ++q)
                chain_next<DT>(ch[q], c, sm->rows[j + k][q]);
        }
#pragma unroll
        for (int q = 0; q < NP; ++q)
            ch[q].template finish<kTanNormDegree(G)>(pk[q]);
    }
};

// The launch's steps on a strip tile: each chunk of table entries is staged by
// bulk copy (double buffered, bounded waits), expanded into the row table,
// then stepped in groups of G aligned to absolute step indices (ragged ends one
// step at a time, as run_step_groups).  G = 1: every step alone (series degrees
// DC, DS).  G >= 2: tan-normalised groups of tan degree DT, as on the
// contiguous tiles.
template <int SCHEME, int G, int DC, int DS, int DT, int NP>
__device__ __forceinline__ bool run_strip(const ReqDesc &R, StripSmem &sm, uint64_t *bars, int *err,
                                          const StripThread<SCHEME, NP> &th,
                                          const float (&pyh)[2 * NP],
                                          const float (&pyl)[2 * NP], MixedPack (&pk)[NP])
{
    constexpr bool kTan = G >= 2;
    using E = StripEntry<SCHEME>;
    using St = Stager<E, kStripStage>;
    constexpr int GA = G > St::kAlign ? G : St::kAlign;  // staging starts on a group and 16 bytes
    static_assert(St::kCh % GA == 0, "chunks hold whole groups");
    const int64_t b_al = R.step_begin & ~static_cast<int64_t>(GA - 1);
    if (!table_range_ok(R, b_al, err))
        return false;
    St st{&sm.stage[0][0], bars, static_cast<const E *>(R.table) + b_al, R.step_end - b_al, 0};
    st.withhold_first = R.withhold_first_copy;
    if (R.step_end <= R.step_begin)
        st.nsteps = 0;
    st.nchunks = static_cast<int>((st.nsteps + St::kCh - 1) / St::kCh);
    if (threadIdx.x == 0) {
        if (st.nchunks > 0) st.issue(0);
        if (st.nchunks > 1) st.issue(1);
    }
    const auto one = [&](int j) {
        if constexpr (kTan)
            th.template single_tan<G, DT>(pk, j);
        else
            th.template single<DC, DS>(pk, j);
    };
    for (int c = 0; c < st.nchunks; ++c) {
        const bool ok = mbar_wait_bounded(&bars[c & 1], (c >> 1) & 1);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0)
                st.on_timeout(c, err);
            return false;
        }
        const E *tb = st.stage(c);
        const int len = st.chunk_len(c);
        // the row table of this chunk, from dt P_y = dt p_hi + (dt A_y + dt p_lo)
        for (int j = threadIdx.x; j < len; j += blockDim.x) {
            const E a = tb[j];
            float dx = 0.0f;
            sm.ax[j] = a.x;
            if constexpr (SCHEME == 2) {
                sm.dy[j] = a.w;
                dx = a.z;
            }
#pragma unroll
            for (int q = 0; q < NP; ++q) {
                const float y0 = __fadd_rn(pyh[2 * q], __fadd_rn(a.y, pyl[2 * q]));
                const float y1 = __fadd_rn(pyh[2 * q + 1], __fadd_rn(a.y, pyl[2 * q + 1]));
                if constexpr (kTan)
                    sm.rows[j][q] = strip_row_tan<SCHEME, DT>(y0, y1, dx);
                else
                    sm.rows[j][q] = strip_row<SCHEME, DC, DS>(y0, y1, dx);
            }
        }
        __syncthreads();  // the table is built and stage c & 1 is free again
        if (threadIdx.x == 0 && c + 2 < st.nchunks)
            st.issue(c + 2);
        // entries before step_begin - b_al belong to earlier launches
        int j = c == 0 ? static_cast<int>(R.step_begin - b_al) : 0;
        if constexpr (G == 1) {
#pragma unroll 2
            for (; j < len; ++j)
                one(j);
        } else {
            for (; j < len && (j & (G - 1)) != 0; ++j)  // ragged start
                one(j);
#pragma unroll kStripGroupUnroll
            for (; j + G <= len; j += G)
                th.template group_tan<G, DT>(pk, j);
            for (; j < len; ++j)  // ragged end (last chunk only)
                one(j);
        }
        __syncthreads();  // everyone is done with the row table
    }
    return true;
}

// Block-uniform dispatch of a strip's steps: tan-normalised groups on (G, DT);
// single steps on the series level (DC, DS).
template <int SCHEME, int DC, int DS, int NP>
__device__ __forceinline__ bool strip_level_steps(const ReqDesc &R, StripSmem &sm, uint64_t *bars,
                                                  int *err, const StripThread<SCHEME, NP> &th,
                                                  const float (&pyh)[2 * NP],
                                                  const float (&pyl)[2 * NP], MixedPack (&pk)[NP])
{
    return run_strip<SCHEME, 1, DC, DS, 0>(R, sm, bars, err, th, pyh, pyl, pk);
}

template <int SCHEME, int L, int NP>
__device__ __forceinline__ bool strip_level(const ReqDesc &R, StripSmem &sm, uint64_t *bars,
                                            int *err, const StripThread<SCHEME, NP> &th,
                                            const float (&pyh)[2 * NP],
                                            const float (&pyl)[2 * NP], MixedPack (&pk)[NP])
{
    if constexpr (L + 1 < kNumLevels) {
        if (R.level != L)
            return strip_level<SCHEME, L + 1>(R, sm, bars, err, th, pyh, pyl, pk);
    }
    return strip_level_steps<SCHEME, kLevelsF32[L].dc, kLevelsF32[L].ds>(R, sm, bars, err, th,
                                                                         pyh, pyl, pk);
}

template <int SCHEME, int G, int I, int NP>
__device__ __forceinline__ bool strip_tan(const ReqDesc &R, StripSmem &sm, uint64_t *bars,
                                          int *err, const StripThread<SCHEME, NP> &th,
                                          const float (&pyh)[2 * NP],
                                          const float (&pyl)[2 * NP], MixedPack (&pk)[NP])
{
    constexpr int DT = kTanDegrees[I];
    if constexpr (I + 1 < kNumTanDegrees) {
        if (R.tdeg != DT)
            return strip_tan<SCHEME, G, I + 1>(R, sm, bars, err, th, pyh, pyl, pk);
    }
    return run_strip<SCHEME, G, 0, 0, DT>(R, sm, bars, err, th, pyh, pyl, pk);
}

template <int SCHEME, int NP>
__device__ __forceinline__ bool strip_steps(const ReqDesc &R, StripSmem &sm, uint64_t *bars,
                                            int *err, const StripThread<SCHEME, NP> &th,
                                            const float (&pyh)[2 * NP],
                                            const float (&pyl)[2 * NP], MixedPack (&pk)[NP])
{
    if (R.group == kGroupMax)
        return strip_tan<SCHEME, kGroupMax, 0>(R, sm, bars, err, th, pyh, pyl, pk);
    if (R.group == 8)
        return strip_tan<SCHEME, 8, 0>(R, sm, bars, err, th, pyh, pyl, pk);
    if (R.group == 4)
        return strip_tan<SCHEME, 4, 0>(R, sm, bars, err, th, pyh, pyl, pk);
    if (R.group == 2)
        return strip_tan<SCHEME, 2, 0>(R, sm, bars, err, th, pyh, pyl, pk);
    return strip_level<SCHEME, 0>(R, sm, bars, err, th, pyh, pyl, pk);
}

// A strip tile of NP packs per thread (2 NP rows: 4 normally, 2 for the strips
// that split a launch's last wave, see ReqDesc::strip_h).
template <int SCHEME, int NP>
__device__ void body_strip(const ReqDesc &R, int tile, unsigned char *smem, uint64_t *bars,
                           int *err)
{
    constexpr int H = 2 * NP;  // rows of the strip
    StripSmem &sm = *reinterpret_cast<StripSmem *>(smem);
    const int tid = threadIdx.x;
    const int ncb = R.nx / kStripThreads;
    const int rb = tile / ncb, cb = tile - rb * ncb;
    const int64_t row_first = R.strip_row0 + static_cast<int64_t>(rb) * H;
    const int64_t col = static_cast<int64_t>(cb) * kStripThreads + tid;
    const double vs = R.valley > 0 ? 1.0 : -1.0;
    float4 *hi_plane = static_cast<float4 *>(R.state);
    float4 *lo_plane = hi_plane + R.n_points;
    // valley K- is stepped as K+ on -P: the table holds -dt*A, here -dt*p
    const double px = grid_node(R.px_min, R.hx, col);
    const double tx = vs * (R.dt * px);
    StripThread<SCHEME, NP> th;
    th.pxh = static_cast<float>(tx);
    th.pxl = static_cast<float>(tx - static_cast<double>(th.pxh));
    th.sm = &sm;
    float pyh[H], pyl[H];
    MixedPoint pt[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
        const int64_t row = row_first + k;
        const bool valid = row < R.ny;  // the last strip of a grid may hang over its end
        const int64_t idx = row * R.nx + col;
        const double py = grid_node(R.py_min, R.hy, R.row0 + row);
        const double ty = vs * (R.dt * py);
        pyh[k] = static_cast<float>(ty);
        pyl[k] = static_cast<float>(ty - static_cast<double>(pyh[k]));
        pt[k].pxh = th.pxh; pt[k].pxl = th.pxl; pt[k].pyh = pyh[k]; pt[k].pyl = pyl[k];
        if (R.fresh || !valid) {
            double ar = 1.0, ai = 0.0, br = 0.0, bi = 0.0;  // identity column
            if (!R.init_identity)
                initial_spinor(px + R.a_in[0], py + R.a_in[1], vs, ar, ai, br, bi);
            pt[k].ar = static_cast<float>(ar);
            pt[k].lar = static_cast<float>(ar - static_cast<double>(pt[k].ar));
            pt[k].ai = static_cast<float>(ai);
            pt[k].lai = static_cast<float>(ai - static_cast<double>(pt[k].ai));
            pt[k].br = static_cast<float>(br);
            pt[k].lbr = static_cast<float>(br - static_cast<double>(pt[k].br));
            pt[k].bi = static_cast<float>(bi);
            pt[k].lbi = static_cast<float>(bi - static_cast<double>(pt[k].bi));
        } else {
            const float4 h = hi_plane[idx], l = lo_plane[idx];
            pt[k].ar = h.x; pt[k].ai = h.y; pt[k].br = h.z; pt[k].bi = h.w;
            pt[k].lar = l.x; pt[k].lai = l.y; pt[k].lbr = l.z; pt[k].lbi = l.w;
        }
    }
    MixedPack pk[NP];
#pragma unroll
    for (int q = 0; q < NP; ++q)
        pk[q] = pack_points(pt[2 * q], pt[2 * q + 1]);
    const bool ok = strip_steps(R, sm, bars, err, th, pyh, pyl, pk);
#pragma unroll
    for (int q = 0; q < NP; ++q)
        unpack_points(pk[q], pt[2 * q], pt[2 * q + 1]);
    if (!ok)
        return;

    float2 *red = reinterpret_cast<float2 *>(smem);  // the staging memory is free now
#pragma unroll
    for (int k = 0; k < H; ++k) {
        const int64_t row = row_first + k;
        const int64_t idx = row * R.nx + col;
        float2 c = make_float2(0.0f, 0.0f);
        if (row < R.ny) {
            if (R.store_state) {
                hi_plane[idx] = make_float4(pt[k].ar, pt[k].ai, pt[k].br, pt[k].bi);
                lo_plane[idx] = make_float4(pt[k].lar, pt[k].lai, pt[k].lbr, pt[k].lbi);
            }
            if (R.project) {
                const SpinorDF v{pt[k].ar, pt[k].lar, pt[k].ai, pt[k].lai,
                                 pt[k].br, pt[k].lbr, pt[k].bi, pt[k].lbi};
                c = store_point<1>(R.map, idx, project_node<1>(R, col, row, v));
            }
        }
        if (R.project)
            red[k * kGranule + tid] = c;
    }
    if (R.project)  // granule of strip row k: row (row_first + k), columns from cb * 256
        granule_sums(red, H, R.partials, (R.n_points + kGranule - 1) / kGranule,
                     [&](int g) { return (row_first + g) * ncb + cb; });
}

template <int SCHEME, int NP>
__global__ void __launch_bounds__(kStripThreads, kMixedMinBlocks)
    evolve_strip_kernel(const __grid_constant__ EvolveArgs args)
{
    __shared__ __align__(128) unsigned char smem[sizeof(StripSmem)];
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
    body_strip<SCHEME, NP>(R, tile, smem, bars, R.err);
}

}  // namespace

#define DSP_CAT4_(a, b, c, d) a##b##c##d
#define DSP_CAT4(a, b, c, d) DSP_CAT4_(a, b, c, d)
#define DSP_STRIP_FN(base) DSP_CAT4(base, _s, DSP_STRIP_SCHEME, DSP_CAT4(_np, DSP_STRIP_NP, , ))

cudaError_t DSP_STRIP_FN(strip_ctas_per_sm)(int *ctas)
{
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        ctas, evolve_strip_kernel<DSP_STRIP_SCHEME, DSP_STRIP_NP>, kStripThreads, 0);
}

cudaError_t DSP_STRIP_FN(launch_evolve_strip)(const EvolveArgs &args, cudaStream_t stream)
{
    if (args.nreq <= 0 || args.total_tiles <= 0)
        return cudaSuccess;
    evolve_strip_kernel<DSP_STRIP_SCHEME, DSP_STRIP_NP>
        <<<args.total_tiles, kStripThreads, 0, stream>>>(args);
    return cudaGetLastError();
}

}  // namespace dsp
