// dsp_device.cuh -- device code shared by the kernels of the split-operator
// massless-Dirac solver (sm_103a; not installed).  The kernels themselves are in
// dsp_mixed.cu (FP32_MIXED, contiguous tiles), dsp_strip.cu (FP32_MIXED, row
// strips) and dsp_kernels.cu (FP64, projection, density, time segments), compiled
// as separate translation units.
//
// Method (arXiv 1607.03062):
//   Sec. II Eq. (free_spin1..4)  initial state v(p + A_in), normalised;
//   Sec. III Eq. (ev_op_dt)      product of N one-step operators, in time order;
//   Sec. III Eq. (approx_time)   step n uses P_n = p + A(t_i + (n + 1/2) dt);
//   Sec. III closed form         U_n = cos(theta) I - i sin(theta) valley sigma.P/|P|,
//                                theta = dt |P_n|;
//   Sec. II Eq. (pair_prod_homo) |c+|^2 = |u(p + A_out)^dag psi|^2, summed to n.
//
// GB300 design (one CTA = one tile of 1024 momenta; FP32-mixed: 256 threads x 4
// spinors, FP64: 512 threads x 2 spinors):
//   * the spinors stay in registers across all steps of a launch: one 16-byte
//     read and one write per spinor plane per launch;
//   * A(t) is staged in shared memory in 16 KB chunks (2048 FP32_MIXED steps,
//     1024 FP64 ones) by 1-D bulk copies (cp.async.bulk) completing on an
//     mbarrier, double buffered, so the step loop reads each entry with one
//     broadcast shared-memory load;
//   * cos(theta) - 1 and sin(theta)/theta are evaluated as their Taylor series
//     in x = theta^2 = |dt P|^2 (no square root, no sin/cos call): the degree is
//     chosen per request on the host from theta_max so truncation stays below
//     the working precision;
//   * FP32_MIXED: dt*p is split into hi + lo (two floats, the momentum of every
//     point to ~1e-16 relative), dt*A(t_n) is one float per step, and
//     P_n = p_hi + (A_n + p_lo): the FP32 roundings of P then change from step
//     to step with A instead of shifting every step's momentum by the same
//     amount, and the first one is at A's scale, not P's;
//   * FP32_MIXED: the spinor is stored as hi + lo and each update adds the
//     increment (U - I) psi with a Fast2Sum, so the FP32 rounding of psi does not
//     random-walk over 1e5 steps; every scheme multiplies 2 to 16 steps into one
//     SU(2) matrix first, so the compensated update is paid once per group, and
//     two momenta share each packed FP32x2 instruction;
//   * the projection and the per-tile partial sums of |c+|^2 are fused into the
//     last launch; partial sums use a fixed pairwise tree, so the density is
//     bitwise reproducible and independent of the batch a request ran in.
// No tensor cores: the work is 2x2 complex arithmetic per momentum.

#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "dsp_df.cuh"
#include "dsp_internal.h"

namespace dsp {
namespace {

// ---------------------------------------------------------------------------
// mbarrier + bulk copy (inline PTX)
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// Global -> shared bulk copy; dst, src 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void *dst, const void *src, uint32_t bytes,
                                          uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Waits for the phase with the given parity; gives up after kWaitLimitNs.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const unsigned long long t0 = global_ns();
    while (true) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (global_ns() - t0 > kWaitLimitNs)
            return false;
    }
}

// ---------------------------------------------------------------------------
// Taylor series in x = theta^2 (written from the power series of cos and sin)
//   cos(theta) - 1    = sum_{k>=1} (-x)^k / (2k)!
//   sin(theta)/theta  = sum_{k>=0} (-x)^k / (2k+1)!
// ---------------------------------------------------------------------------

template <int N>
__host__ __device__ constexpr double inv_factorial()
{
    if constexpr (N <= 1)
        return 1.0;
    else
        return inv_factorial<N - 1>() / static_cast<double>(N);
}

// Horner tail sum_{k=K..D} c_k x^(k-K) with c_k = (-1)^k / (2k + ODD)!; every
// coefficient is a compile-time constant rounded once to T.
template <typename T, int D, int K, int ODD>
__device__ __forceinline__ T horner(T x)
{
    constexpr T c = static_cast<T>(((K & 1) ? -1.0 : 1.0) * inv_factorial<2 * K + ODD>());
    if constexpr (K == D)
        return c;
    else
        return fma(horner<T, D, K + 1, ODD>(x), x, c);
}

template <int D>
__device__ __forceinline__ double cos_f64(double x)
{
    return horner<double, D, 0, 0>(x);
}
template <int D>
__device__ __forceinline__ double sinc_f64(double x)
{
    return horner<double, D, 0, 1>(x);
}

// ---------------------------------------------------------------------------
// Per-point set-up shared by both precisions (all FP64, once per launch)
// ---------------------------------------------------------------------------

// Cell-centred node p = p_min + (i + 1/2) h, without contraction.
__device__ __forceinline__ double grid_node(double lo, double h, int64_t i)
{
    return __dadd_rn(lo, __dmul_rn(static_cast<double>(i) + 0.5, h));
}

// Negative-energy spinor v(P) of valley * sigma.P, normalised (Sec. II Eq.
// (free_spin1..4)); at P = 0 the limit P -> (0+, 0).
__device__ __forceinline__ void initial_spinor(double Px, double Py, double sgn, double &ar,
                                               double &ai, double &br, double &bi)
{
    const double r = 0.70710678118654752440;
    const double E = sqrt(Px * Px + Py * Py);
    if (E > 0.0) {
        ar = sgn * (-Px / E) * r;
        ai = sgn * (Py / E) * r;
    } else {
        ar = -sgn * r;
        ai = 0.0;
    }
    br = r;
    bi = 0.0;
}

// |u(P_out)^dag psi|^2 with u = [1, valley (Px + i Py)/E]/sqrt(2); 0 at P_out = 0.
// FP64; used only for the rare points whose |P_out| is too small for the
// double-float form below.
__device__ __forceinline__ double project_point(double Px, double Py, double sgn, double ar,
                                                double ai, double br, double bi)
{
    const double E = sqrt(Px * Px + Py * Py);
    if (!(E > 0.0))
        return 0.0;
    const double wr = sgn * Px / E, wi = -sgn * Py / E;  // valley * conj(Px + i Py)/E
    const double cr = ar + (wr * br - wi * bi);
    const double ci = ai + (wr * bi + wi * br);
    return 0.5 * (cr * cr + ci * ci);
}

// ---------------------------------------------------------------------------
// The projection |c+|^2 = |u(P_out)^dag psi|^2 in double-float FP32 arithmetic.
//
// GB300 issues FP64 at about 1/64 of its FP32 rate, and an FP64 projection (a
// square root and two divisions per point) would make a projection-only launch
// FP64-bound at a small fraction of HBM speed.  Here every quantity is an
// unevaluated pair hi + lo of floats (about 48 significant bits): products are
// split exactly with FMA, the large terms of c+ are summed with TwoSum, so
// |c+|^2 comes out to ~1e-14 absolute; only its conversion to double and the
// tile tree use FP64.  The node P_out = p + A_out (valley-signed) comes from a
// per-grid table of hi/lo pairs built on the host in FP64.  Written from the
// definitions (TwoSum, the FMA product split, one Newton step for 1/sqrt);
// all operations are non-contracting intrinsics, so every kernel that calls it
// gets the same bits.
// ---------------------------------------------------------------------------

// Points with E^2 = |P_out|^2 below this (|P_out| < 2^-45 eV) take the FP64
// form: their squares would lose bits near the bottom of the float range.
constexpr float kProjTinyE2 = 0x1p-90f;

// |c+|^2 = oh + ol for the node s P_out = (xh + xl, yh + yl) (s = valley) and
// the spinor a = (ar, ai), b = (br, bi), each component hi + lo:
//   c+ = (a + conj(w) b)/sqrt(2),  w = s (P_x + i P_y)/|P|,
//   cr = ar + wr br + wi bi,  ci = ai + wr bi - wi br.
// Returns false (and leaves oh, ol unset) when E^2 < kProjTinyE2.
__device__ __forceinline__ bool project_df(float xh, float xl, float yh, float yl, float arh,
                                           float arl, float aih, float ail, float brh, float brl,
                                           float bih, float bil, float &oh, float &ol)
{
    // E^2 = Px^2 + Py^2 to ~2^-46
    const float x2 = __fmul_rn(xh, xh);
    const float x2e = __fmaf_rn(__fadd_rn(xh, xh), xl, __fmaf_rn(xh, xh, -x2));
    const float y2 = __fmul_rn(yh, yh);
    const float y2e = __fmaf_rn(__fadd_rn(yh, yh), yl, __fmaf_rn(yh, yh, -y2));
    float sh, se;
    two_sum(x2, y2, sh, se);
    se = __fadd_rn(se, __fadd_rn(x2e, y2e));
    if (!(sh >= kProjTinyE2))
        return false;
    // r = 1/E = r0 + rc: one Newton step r0 (1 - t/2) from the FP32 estimate r0,
    // with t = E^2 r0^2 - 1 evaluated to ~2^-46 (p - 1 is exact: p is near 1)
    const float r0 = rsqrtf(sh);
    const float q = __fmul_rn(r0, r0), qe = __fmaf_rn(r0, r0, -q);
    const float p = __fmul_rn(sh, q), pe = __fmaf_rn(sh, q, -p);
    const float t = __fadd_rn(__fadd_rn(p, -1.0f), __fmaf_rn(sh, qe, __fmaf_rn(se, q, pe)));
    const float rc = __fmul_rn(__fmul_rn(-0.5f, r0), t);
    // w = (wr + wre) + i (wi + wie) = s P / E
    const float wr = __fmul_rn(xh, r0);
    const float wre = __fmaf_rn(xh, rc, __fmaf_rn(xl, r0, __fmaf_rn(xh, r0, -wr)));
    const float wi = __fmul_rn(yh, r0);
    const float wie = __fmaf_rn(yh, rc, __fmaf_rn(yl, r0, __fmaf_rn(yh, r0, -wi)));
    // cr: the three large terms ar, wr br, wi bi exactly (split products, TwoSum),
    // then the small ones (lo parts, product errors, cross terms) in FP32
    float crh, crl;
    {
        const float p1 = __fmul_rn(wr, brh), e1 = __fmaf_rn(wr, brh, -p1);
        const float p2 = __fmul_rn(wi, bih), e2 = __fmaf_rn(wi, bih, -p2);
        float t1, te, ce;
        two_sum(p1, p2, t1, te);
        two_sum(arh, t1, crh, ce);
        float l = __fadd_rn(__fadd_rn(ce, te), __fadd_rn(arl, __fadd_rn(e1, e2)));
        l = __fmaf_rn(wre, brh, __fmaf_rn(wr, brl, l));
        crl = __fmaf_rn(wie, bih, __fmaf_rn(wi, bil, l));
    }
    float cih, cil;
    {
        const float p3 = __fmul_rn(wr, bih), e3 = __fmaf_rn(wr, bih, -p3);
        const float p4 = __fmul_rn(-wi, brh), e4 = __fmaf_rn(-wi, brh, -p4);
        float t2, te, ce;
        two_sum(p3, p4, t2, te);
        two_sum(aih, t2, cih, ce);
        float l = __fadd_rn(__fadd_rn(ce, te), __fadd_rn(ail, __fadd_rn(e3, e4)));
        l = __fmaf_rn(wre, bih, __fmaf_rn(wr, bil, l));
        cil = __fmaf_rn(-wie, brh, __fmaf_rn(-wi, brl, l));
    }
    // |c|^2 = cr^2 + ci^2 after renormalising each pair (cancellation can leave
    // the lo part as large as the hi part)
    float ch, cl, dh, dl;
    two_sum(crh, crl, ch, cl);
    two_sum(cih, cil, dh, dl);
    const float c2 = __fmul_rn(ch, ch);
    const float c2e = __fmaf_rn(__fadd_rn(ch, ch), cl, __fmaf_rn(ch, ch, -c2));
    const float d2 = __fmul_rn(dh, dh);
    const float d2e = __fmaf_rn(__fadd_rn(dh, dh), dl, __fmaf_rn(dh, dh, -d2));
    float nh, ne;
    two_sum(c2, d2, nh, ne);
    ne = __fadd_rn(ne, __fadd_rn(c2e, d2e));
    oh = __fmul_rn(0.5f, nh);  // exact scalings
    ol = __fmul_rn(0.5f, ne);
    return true;
}

// |c+|^2 in FP32 (FP32_MIXED, whose map is a float): from the hi parts of the
// node and of the spinor, 1/|P| from rsqrtf and one Newton step.  The error is
// below ~4e-7 |c+| (the FP32 rounding of the products around the cancellation in
// a + conj(w) b), about the size of the float map's own rounding.  Returns false
// when |P_out|^2 < 1e-30.
__device__ __forceinline__ bool project_f32(float x, float y, float ar, float ai, float br,
                                            float bi, float &out)
{
    const float e2 = __fmaf_rn(x, x, __fmul_rn(y, y));
    if (!(e2 >= 1e-30f))
        return false;
    float r = rsqrtf(e2);
    r = __fmaf_rn(__fmul_rn(0.5f, r), __fmaf_rn(-e2, __fmul_rn(r, r), 1.0f), r);  // Newton
    const float wr = __fmul_rn(x, r), wi = __fmul_rn(y, r);
    const float cr = __fmaf_rn(wr, br, __fmaf_rn(wi, bi, ar));
    const float ci = __fmaf_rn(wr, bi, __fmaf_rn(-wi, br, ai));
    out = __fmul_rn(0.5f, __fmaf_rn(cr, cr, __fmul_rn(ci, ci)));
    return true;
}

// |c+|^2 of the point in column col and row row of the grid (global row row0 +
// row) as a double-float pair: FP32_MIXED (PREC 1) in FP32 (project_f32), FP64
// (PREC 0) in double-float (project_df); FP64 for the points whose |P_out| is too
// small for either (their doubles are formed only there).
struct SpinorDF {
    float arh, arl, aih, ail, brh, brl, bih, bil;
};

// The same with the node table's entries of the column (cx) and row (cy) given.
template <int PREC>
__device__ __forceinline__ float2 project_node_at(const ReqDesc &R, float2 cx, float2 cy,
                                                  int64_t col, int64_t row, const SpinorDF &v)
{
    if constexpr (PREC == 1) {
        float o;
        if (project_f32(cx.x, cy.x, v.arh, v.aih, v.brh, v.bih, o))
            return make_float2(o, 0.0f);
    } else {
        float oh, ol;
        if (project_df(cx.x, cx.y, cy.x, cy.y, v.arh, v.arl, v.aih, v.ail, v.brh, v.brl, v.bih,
                       v.bil, oh, ol))
            return make_float2(oh, ol);
    }
    const double vs = R.valley > 0 ? 1.0 : -1.0;
    const double px = grid_node(R.px_min, R.hx, col);
    const double py = grid_node(R.py_min, R.hy, R.row0 + row);
    const double c2 = project_point(px + R.a_out[0], py + R.a_out[1], vs,
                                    f32_to_f64(v.arh) + f32_to_f64(v.arl),
                                    f32_to_f64(v.aih) + f32_to_f64(v.ail),
                                    f32_to_f64(v.brh) + f32_to_f64(v.brl),
                                    f32_to_f64(v.bih) + f32_to_f64(v.bil));
    float h, l;
    split_f64(c2, h, l);
    return make_float2(h, l);
}

template <int PREC>
__device__ __forceinline__ float2 project_node(const ReqDesc &R, int64_t col, int64_t row,
                                               const SpinorDF &v)
{
    return project_node_at<PREC>(R, R.nodes_out[col], R.nodes_out[R.nx + row], col, row, v);
}

// The map value of a point and its term in the density sum, from |c+|^2 = c.x +
// c.y: FP32_MIXED stores the float nearest the pair and sums the pair itself;
// FP64 stores the double and sums that double (split into a pair), so that the
// density is the sum of the FP64 map's values.
template <int PREC>
__device__ __forceinline__ float2 store_point(void *map, int64_t idx, float2 c)
{
    if constexpr (PREC == 1) {
        if (map)
            static_cast<float *>(map)[idx] = __fadd_rn(c.x, c.y);
        return c;
    } else {
        const double d = df_to_f64(c.x, c.y);
        if (map)
            static_cast<double *>(map)[idx] = d;
        float h, l;
        split_f64(d, h, l);
        return make_float2(h, l);
    }
}

// Locates the request tile b (by default the CTA's own) belongs to (requests are
// sorted by tile_begin).
__device__ __forceinline__ int find_request(const EvolveArgs &a,
                                            int b = static_cast<int>(blockIdx.x))
{
    int lo = 0, hi = a.nreq - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.r[mid].tile_begin <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------
// Table staging: chunk c of the launch goes to stage c & 1 of shared memory.
// ---------------------------------------------------------------------------

constexpr int kStageBytes = 16384;  // per stage; two stages per CTA

// Tuning constants: unroll factors of the loop over groups of two steps and of
// the chain inside a step group, and spinors per thread of the FP32-mixed kernel
// (even: the steps run on FP32x2 pairs; a CTA always owns one 1024-point tile).
#ifndef DSP_PAIR_UNROLL
#define DSP_PAIR_UNROLL 2
#endif
#ifndef DSP_MIXED_SPT
#define DSP_MIXED_SPT 4
#endif
#ifndef DSP_MIXED_MINB
#define DSP_MIXED_MINB 2
#endif
#ifndef DSP_GROUP_UNROLL
#define DSP_GROUP_UNROLL 8
#endif
constexpr int kPairUnroll = DSP_PAIR_UNROLL;
constexpr int kGroupUnroll = DSP_GROUP_UNROLL;  // chain loop inside one group (>= G - 2: whole)
constexpr int kMixedSpt = DSP_MIXED_SPT;
constexpr int kMixedThreads = kTilePoints / kMixedSpt;
constexpr int kMixedMinBlocks = DSP_MIXED_MINB;  // resident CTAs per SM the registers allow
constexpr int kF64Threads = kThreads;
static_assert(kTilePoints % kMixedSpt == 0, "a CTA owns one whole tile");
static_assert(kMixedSpt % 2 == 0, "FP32x2 pairs of spinors");

// MAGNUS4 table entries: the Gauss-point mean (dt*Abar, valley-signed) and the
// commutator factor D = -(sqrt(3)/6) dt (A2 - A1) (valley-signed).  FP32_MIXED:
// one float4 (Abar_x, Abar_y, D_x, D_y).
struct F64G2 {
    double2 a;  // Abar
    double2 d;  // D
};

// Bounds-check builds (-DDSP_BOUNDS_CHECK) verify, uniformly per CTA, that the
// table entries a launch stages, [first, step_end), lie inside the table (the
// copy's rounding up to 16 bytes stays in the allocation's padding); a bad range
// sets kErrBounds and the launch does nothing.  Otherwise a no-op.
__device__ __forceinline__ bool table_range_ok(const ReqDesc &R, int64_t first, int *err)
{
#ifdef DSP_BOUNDS_CHECK
    const bool ok = first >= 0 && R.step_end >= R.step_begin &&
                    (R.step_end == R.step_begin || R.step_end <= R.table_steps);
    if (!ok && threadIdx.x == 0)
        atomicOr(err, kErrBounds);
    return ok;
#else
    (void)R;
    (void)first;
    (void)err;
    return true;
#endif
}

// Bounds-check builds verify a CTA's tile index; a bad one sets kErrBounds.
__device__ __forceinline__ bool tile_ok(const ReqDesc &R, int tile, int *err)
{
#ifdef DSP_BOUNDS_CHECK
    const bool ok = tile >= 0 && tile < R.n_tiles;
    if (!ok && threadIdx.x == 0)
        atomicOr(err, kErrBounds);
    return ok;
#else
    (void)R;
    (void)tile;
    (void)err;
    return true;
#endif
}

// Stages table entries [base, base + nsteps) in chunks of kCh.  A 1-D bulk copy
// must start and end on 16-byte boundaries: base is a multiple of kAlign entries
// (16 bytes), every chunk is a multiple of kAlign, and the last copy is rounded
// up to whole 16 bytes, which stays inside the table's allocation (the library
// pads it to a multiple of 16 bytes).
template <typename E, int kBytes = kStageBytes>
struct Stager {
    unsigned char *smem;
    uint64_t *bars;
    const E *table;  // entry base is element 0 of chunk 0
    int64_t nsteps;
    int nchunks;
    int withhold_first = 0;  // test hook (ReqDesc::withhold_first_copy)
    static constexpr int kCh = kBytes / static_cast<int>(sizeof(E));
    static constexpr int kAlign = sizeof(E) >= 16 ? 1 : static_cast<int>(16 / sizeof(E));
    static_assert(16 % sizeof(E) == 0 || sizeof(E) % 16 == 0, "entries tile 16 bytes");
    static_assert(kCh % kAlign == 0, "chunks start on 16-byte boundaries");

    __device__ __forceinline__ const E *stage(int c) const
    {
        return reinterpret_cast<const E *>(smem + (c & 1) * kBytes);
    }
    __device__ __forceinline__ int chunk_len(int c) const
    {
        const int64_t rem = nsteps - static_cast<int64_t>(c) * kCh;
        return rem < kCh ? static_cast<int>(rem) : kCh;
    }
    __device__ __forceinline__ void issue(int c) const  // one thread
    {
        const uint32_t bytes = (static_cast<uint32_t>(chunk_len(c)) * sizeof(E) + 15u) & ~15u;
        mbar_arrive_expect_tx(&bars[c & 1], bytes);
        if (c == 0 && withhold_first)
            return;  // the phase cannot complete: its waiters time out
        bulk_load(smem + (c & 1) * kBytes, table + static_cast<int64_t>(c) * kCh, bytes,
                  &bars[c & 1]);
    }
    // After the wait for chunk c timed out (one thread): flags the error and gives
    // the copy of chunk c + 1, if it was issued, a bounded chance to land first.
    __device__ __forceinline__ void on_timeout(int c, int *err) const
    {
        atomicOr(err, kErrTimeout);
        if (c + 1 < nchunks)
            (void)mbar_wait_bounded(&bars[(c + 1) & 1], ((c + 1) >> 1) & 1);
    }
};

// Runs the launch's steps with the table streamed through shared memory; STEP
// is called as step(entry) for every step in order.  Returns false (and flags
// err) if a staging wait timed out.
template <typename E, typename StepFn>
__device__ __forceinline__ bool run_steps(const ReqDesc &R, unsigned char *smem, uint64_t *bars,
                                          int *err, StepFn step)
{
    const int64_t b_al = R.step_begin & ~static_cast<int64_t>(Stager<E>::kAlign - 1);
    if (!table_range_ok(R, b_al, err))
        return false;
    Stager<E> st{smem, bars, static_cast<const E *>(R.table) + b_al, R.step_end - b_al, 0};
    st.withhold_first = R.withhold_first_copy;
    if (R.step_end <= R.step_begin)
        st.nsteps = 0;
    st.nchunks = static_cast<int>((st.nsteps + Stager<E>::kCh - 1) / Stager<E>::kCh);
    if (threadIdx.x == 0) {
        if (st.nchunks > 0) st.issue(0);
        if (st.nchunks > 1) st.issue(1);
    }
    for (int c = 0; c < st.nchunks; ++c) {
        const bool ok = mbar_wait_bounded(&bars[c & 1], (c >> 1) & 1);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0)
                st.on_timeout(c, err);
            return false;
        }
        const E *tb = st.stage(c);
        const int len = st.chunk_len(c);
        // entries before step_begin - b_al belong to earlier launches
#pragma unroll 2
        for (int j = c == 0 ? static_cast<int>(R.step_begin - b_al) : 0; j < len; ++j)
            step(tb[j]);  // shared-memory broadcast
        __syncthreads();  // everyone is done with stage c & 1
        if (threadIdx.x == 0 && c + 2 < st.nchunks)
            st.issue(c + 2);
    }
    return true;
}

// As run_steps, but steps are taken in groups (G j, ..., G j + G - 1) of ABSOLUTE
// step index (a launch that starts or ends inside a group takes those steps one
// by one), so any split of a run at multiples of G meets the same groups.  The
// stages hold whole groups: staging starts at the multiple of G at or below
// step_begin and the stage length is a multiple of G.  GROUP is called as
// group(e) with e the group's G consecutive entries in shared memory.
template <typename E, int G, typename SingleFn, typename GroupFn>
__device__ __forceinline__ bool run_step_groups(const ReqDesc &R, unsigned char *smem,
                                                uint64_t *bars, int *err, SingleFn single,
                                                GroupFn group)
{
    static_assert(G >= 2 && (G & (G - 1)) == 0, "group size: a power of two");
    static_assert(Stager<E>::kCh % G == 0, "stages must hold whole groups");
    static_assert(G % Stager<E>::kAlign == 0, "groups start on 16-byte boundaries");
    const int64_t b_al = R.step_begin & ~static_cast<int64_t>(G - 1);
    if (!table_range_ok(R, b_al, err))
        return false;
    Stager<E> st{smem, bars, static_cast<const E *>(R.table) + b_al, R.step_end - b_al, 0};
    st.withhold_first = R.withhold_first_copy;
    if (R.step_end <= R.step_begin)
        st.nsteps = 0;
    st.nchunks = static_cast<int>((st.nsteps + Stager<E>::kCh - 1) / Stager<E>::kCh);
    if (threadIdx.x == 0) {
        if (st.nchunks > 0) st.issue(0);
        if (st.nchunks > 1) st.issue(1);
    }
    for (int c = 0; c < st.nchunks; ++c) {
        const bool ok = mbar_wait_bounded(&bars[c & 1], (c >> 1) & 1);
        if (!__syncthreads_and(ok)) {
            if (threadIdx.x == 0)
                st.on_timeout(c, err);
            return false;
        }
        const E *tb = st.stage(c);
        const int len = st.chunk_len(c);
        // entries before step_begin - b_al belong to earlier launches
        int j = c == 0 ? static_cast<int>(R.step_begin - b_al) : 0;
        for (; j < len && (j & (G - 1)) != 0; ++j)  // ragged start
            single(tb[j]);
        if constexpr (G == 2) {
#pragma unroll kPairUnroll
            for (; j + G <= len; j += G)
                group(tb + j);
        } else {
#pragma unroll 1
            for (; j + G <= len; j += G)
                group(tb + j);
        }
        for (; j < len; ++j)  // ragged end (last stage only)
            single(tb[j]);
        __syncthreads();  // everyone is done with stage c & 1
        if (threadIdx.x == 0 && c + 2 < st.nchunks)
            st.issue(c + 2);
    }
    return true;
}

// ---------------------------------------------------------------------------
// FP32_MIXED state of one momentum (loads and stores; the steps run packed)
// ---------------------------------------------------------------------------

struct MixedPoint {
    float ar, ai, br, bi;      // hi parts of psi = (a, b)
    float lar, lai, lbr, lbi;  // lo parts
    float pxh, pxl, pyh, pyl;  // dt * p as hi + lo
};

// ---------------------------------------------------------------------------
// Packed FP32x2 steps: lane 0 and lane 1 of every float2 belong to two
// different momenta; each lane is rounded as the scalar FP32 operation would
// be, so one instruction issues the arithmetic of two spinors and either lane's
// result is the one-momentum result.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 bc2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 neg2(float2 v) { return make_float2(-v.x, -v.y); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, neg2(b)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

template <int D, int K, int ODD>
__device__ __forceinline__ float2 horner2(float2 x)
{
    constexpr float c = static_cast<float>(((K & 1) ? -1.0 : 1.0) * inv_factorial<2 * K + ODD>());
    if constexpr (K == D)
        return bc2(c);
    else
        return fma2(horner2<D, K + 1, ODD>(x), x, bc2(c));
}

struct MixedPack {
    float2 ar, ai, br, bi, lar, lai, lbr, lbi, pxh, pxl, pyh, pyl;
};

__device__ __forceinline__ MixedPack pack_points(const MixedPoint &u, const MixedPoint &v)
{
    MixedPack p;
    p.ar = make_float2(u.ar, v.ar); p.ai = make_float2(u.ai, v.ai);
    p.br = make_float2(u.br, v.br); p.bi = make_float2(u.bi, v.bi);
    p.lar = make_float2(u.lar, v.lar); p.lai = make_float2(u.lai, v.lai);
    p.lbr = make_float2(u.lbr, v.lbr); p.lbi = make_float2(u.lbi, v.lbi);
    p.pxh = make_float2(u.pxh, v.pxh); p.pxl = make_float2(u.pxl, v.pxl);
    p.pyh = make_float2(u.pyh, v.pyh); p.pyl = make_float2(u.pyl, v.pyl);
    return p;
}

__device__ __forceinline__ void unpack_points(const MixedPack &p, MixedPoint &u, MixedPoint &v)
{
    u.ar = p.ar.x; v.ar = p.ar.y; u.ai = p.ai.x; v.ai = p.ai.y;
    u.br = p.br.x; v.br = p.br.y; u.bi = p.bi.x; v.bi = p.bi.y;
    u.lar = p.lar.x; v.lar = p.lar.y; u.lai = p.lai.x; v.lai = p.lai.y;
    u.lbr = p.lbr.x; v.lbr = p.lbr.y; u.lbi = p.lbi.x; v.lbi = p.lbi.y;
}

// step_coeffs_f32<0> on two momenta at once
template <int DC, int DS>
__device__ __forceinline__ void coeffs_exact2(const MixedPack &p, const float2 &a, float2 &m,
                                              float2 &qr, float2 &qi)
{
    const float2 Px = add2(p.pxh, add2(bc2(a.x), p.pxl));
    const float2 Py = add2(p.pyh, add2(bc2(a.y), p.pyl));
    const float2 x = fma2(Px, Px, mul2(Py, Py));
    m = mul2(horner2<DC, 1, 0>(x), x);
    const float2 sn = horner2<DS, 0, 1>(x);
    qr = mul2(sn, Py);
    qi = mul2(sn, Px);
}

// Compensated update psi <- psi + d, d = (M - I) psi_hi + psi_lo, for
// M - I = [[am + i ai, -Q], [conj(Q), am - i ai]] (ai = 0 for one step).
__device__ __forceinline__ void apply2(MixedPack &p, float2 am, float2 ai, float2 Qr, float2 Qi)
{
    const float2 nai = neg2(ai), nQr = neg2(Qr), nQi = neg2(Qi);
    const float2 dar = fma2(am, p.ar, fma2(nai, p.ai, fma2(nQr, p.br, fma2(Qi, p.bi, p.lar))));
    const float2 dai = fma2(am, p.ai, fma2(ai, p.ar, fma2(nQr, p.bi, fma2(nQi, p.br, p.lai))));
    const float2 dbr = fma2(am, p.br, fma2(ai, p.bi, fma2(Qr, p.ar, fma2(Qi, p.ai, p.lbr))));
    const float2 dbi = fma2(am, p.bi, fma2(nai, p.br, fma2(Qr, p.ai, fma2(nQi, p.ar, p.lbi))));
    float2 t;
    t = add2(p.ar, dar); p.lar = sub2(dar, sub2(t, p.ar)); p.ar = t;
    t = add2(p.ai, dai); p.lai = sub2(dai, sub2(t, p.ai)); p.ai = t;
    t = add2(p.br, dbr); p.lbr = sub2(dbr, sub2(t, p.br)); p.br = t;
    t = add2(p.bi, dbi); p.lbi = sub2(dbi, sub2(t, p.bi)); p.bi = t;
}

// psi <- U psi for one EXACT step, U - I = [[m, -q], [conj(q), m]] (apply_f32<0>).
__device__ __forceinline__ void apply_exact2(MixedPack &p, float2 m, float2 qr, float2 qi)
{
    const float2 nqr = neg2(qr), nqi = neg2(qi);
    const float2 dar = fma2(m, p.ar, fma2(nqr, p.br, fma2(qi, p.bi, p.lar)));
    const float2 dai = fma2(m, p.ai, fma2(nqr, p.bi, fma2(nqi, p.br, p.lai)));
    const float2 dbr = fma2(m, p.br, fma2(qr, p.ar, fma2(qi, p.ai, p.lbr)));
    const float2 dbi = fma2(m, p.bi, fma2(qr, p.ai, fma2(nqi, p.ar, p.lbi)));
    float2 t;
    t = add2(p.ar, dar); p.lar = sub2(dar, sub2(t, p.ar)); p.ar = t;
    t = add2(p.ai, dai); p.lai = sub2(dai, sub2(t, p.ai)); p.ai = t;
    t = add2(p.br, dbr); p.lbr = sub2(dbr, sub2(t, p.br)); p.br = t;
    t = add2(p.bi, dbi); p.lbi = sub2(dbi, sub2(t, p.bi)); p.bi = t;
}

// One EXACT step (apply_f32<0> with cm1 = m, q = (qr, qi)).
template <int DC, int DS>
__device__ __forceinline__ void step_exact2(MixedPack &p, const float2 &a)
{
    float2 m, qr, qi;
    coeffs_exact2<DC, DS>(p, a, m, qr, qi);
    apply_exact2(p, m, qr, qi);
}

// One MAGNUS4 step (step_coeffs_f32<2> + apply_f32<2> on two momenta):
// U - I = [[m - i qz, -q], [conj(q), m + i qz]].
template <int DC, int DS>
__device__ __forceinline__ void step_magnus2(MixedPack &p, const float4 &e)
{
    const float2 Px = add2(p.pxh, add2(bc2(e.x), p.pxl));
    const float2 Py = add2(p.pyh, add2(bc2(e.y), p.pyl));
    const float2 nz = fma2(Px, bc2(e.w), neg2(mul2(Py, bc2(e.z))));
    const float2 x = fma2(Px, Px, fma2(Py, Py, mul2(nz, nz)));
    const float2 m = mul2(horner2<DC, 1, 0>(x), x);
    const float2 sn = horner2<DS, 0, 1>(x);
    apply2(p, m, neg2(mul2(sn, nz)), mul2(sn, Py), mul2(sn, Px));
}

// ---------------------------------------------------------------------------
// Step groups, written for V = float2 (two momenta per instruction; a V = float
// instantiation performs the same roundings for one) with non-contracting
// intrinsics.
// ---------------------------------------------------------------------------

[[maybe_unused]] __device__ __forceinline__ float vadd(float a, float b) { return __fadd_rn(a, b); }
[[maybe_unused]] __device__ __forceinline__ float vmul(float a, float b) { return __fmul_rn(a, b); }
[[maybe_unused]] __device__ __forceinline__ float vfma(float a, float b, float c)
{
    return __fmaf_rn(a, b, c);
}
[[maybe_unused]] __device__ __forceinline__ float vneg(float a) { return -a; }
[[maybe_unused]] __device__ __forceinline__ float2 vadd(float2 a, float2 b) { return add2(a, b); }
[[maybe_unused]] __device__ __forceinline__ float2 vmul(float2 a, float2 b) { return mul2(a, b); }
[[maybe_unused]] __device__ __forceinline__ float2 vfma(float2 a, float2 b, float2 c)
{
    return fma2(a, b, c);
}
[[maybe_unused]] __device__ __forceinline__ float2 vneg(float2 a) { return neg2(a); }
template <typename V>
__device__ __forceinline__ V vbc(float v);
template <>
[[maybe_unused]] __device__ __forceinline__ float vbc<float>(float v) { return v; }
template <>
[[maybe_unused]] __device__ __forceinline__ float2 vbc<float2>(float v) { return bc2(v); }

template <typename V, int D, int K, int ODD>
__device__ __forceinline__ V vhorner(V x)
{
    constexpr float c = static_cast<float>(((K & 1) ? -1.0 : 1.0) * inv_factorial<2 * K + ODD>());
    if constexpr (K == D)
        return vbc<V>(c);
    else
        return vfma(vhorner<V, D, K + 1, ODD>(x), x, vbc<V>(c));
}

// Coefficient sets of the tan-normalised groups (kTanSeries, kSecSeries) and of
// (1 + y)^(-1/2): c_k = binom(-1/2, k) = prod_{j=1..k} -(2j - 1)/(2j).
struct TanCoef {
    __host__ __device__ static constexpr double at(int k) { return kTanSeries[k]; }
};
struct SecCoef {
    __host__ __device__ static constexpr double at(int k) { return kSecSeries[k]; }
};
struct RsqrtCoef {
    __host__ __device__ static constexpr double at(int k)
    {
        double c = 1.0;
        for (int j = 1; j <= k; ++j)
            c *= -static_cast<double>(2 * j - 1) / static_cast<double>(2 * j);
        return c;
    }
};

// Horner tail sum_{k=K..D} C::at(k) x^(k-K), coefficients rounded once to float.
template <typename V, typename C, int D, int K>
__device__ __forceinline__ V vseries(V x)
{
    constexpr float c = static_cast<float>(C::at(K));
    if constexpr (K == D)
        return vbc<V>(c);
    else
        return vfma(vseries<V, C, D, K + 1>(x), x, vbc<V>(c));
}

// Compensated update psi <- psi + d, d = (M - I) psi_hi + psi_lo, for
// M - I = [[am + i ai, -Q], [conj(Q), am - i ai]]: the operations of apply2.
template <typename Pt, typename V>
__device__ __forceinline__ void apply_group(Pt &p, V am, V ai, V Qr, V Qi)
{
    const V nai = vneg(ai), nQr = vneg(Qr), nQi = vneg(Qi);
    const V dar = vfma(am, p.ar, vfma(nai, p.ai, vfma(nQr, p.br, vfma(Qi, p.bi, p.lar))));
    const V dai = vfma(am, p.ai, vfma(ai, p.ar, vfma(nQr, p.bi, vfma(nQi, p.br, p.lai))));
    const V dbr = vfma(am, p.br, vfma(ai, p.bi, vfma(Qr, p.ar, vfma(Qi, p.ai, p.lbr))));
    const V dbi = vfma(am, p.bi, vfma(nai, p.br, vfma(Qr, p.ai, vfma(nQi, p.ar, p.lbi))));
    V t;
    t = vadd(p.ar, dar); p.lar = vadd(dar, vneg(vadd(t, vneg(p.ar)))); p.ar = t;
    t = vadd(p.ai, dai); p.lai = vadd(dai, vneg(vadd(t, vneg(p.ai)))); p.ai = t;
    t = vadd(p.br, dbr); p.lbr = vadd(dbr, vneg(vadd(t, vneg(p.br)))); p.br = t;
    t = vadd(p.bi, dbi); p.lbi = vadd(dbi, vneg(vadd(t, vneg(p.bi)))); p.bi = t;
}

// STRANG_XY's merged step X(a) Y(b) X(a), 2a = dt Px, b = dt Py, as m = cos b
// cos 2a - 1 and q = sin b + i cos b sin 2a, from small parts only:
// m = cx + cy + cx cy (cx = cos 2a - 1, cy = cos b - 1), sin 2a = Px + (sinc - 1) Px,
// sin b likewise, cos b sin 2a = sin 2a + cy sin 2a.  (Steps taken one at a time,
// G = 1.)
template <int DC, int DS, typename Pt, typename V>
__device__ __forceinline__ void coeffs_strang(const Pt &p, const float2 &a, V &m, V &qr, V &qi)
{
    const V Px = vadd(p.pxh, vadd(vbc<V>(a.x), p.pxl));
    const V Py = vadd(p.pyh, vadd(vbc<V>(a.y), p.pyl));
    const V xx = vmul(Px, Px), xy = vmul(Py, Py);
    const V cx = vmul(vhorner<V, DC, 1, 0>(xx), xx), cy = vmul(vhorner<V, DC, 1, 0>(xy), xy);
    const V sx = vfma(vmul(vhorner<V, DS, 1, 1>(xx), xx), Px, Px);
    qr = vfma(vmul(vhorner<V, DS, 1, 1>(xy), xy), Py, Py);
    qi = vfma(cy, sx, sx);
    m = vfma(cx, cy, vadd(cx, cy));
}

// One STRANG_XY step alone: U - I = [[m, -q], [conj(q), m]].
template <int DC, int DS, typename Pt>
__device__ __forceinline__ void step_strang(Pt &p, const float2 &a)
{
    using V = decltype(p.ar);
    V m, qr, qi;
    coeffs_strang<DC, DS>(p, a, m, qr, qi);
    apply_group(p, m, vbc<V>(0.0f), qr, qi);
}

// ---------------------------------------------------------------------------
// Tan-normalised step groups (EXACT and STRANG_XY, G = 2, 4, 8, 16; MAGNUS4 uses
// the same chain with its sigma_z part, see coeffs_tan_magnus)
//
// Both schemes step with a real diagonal: U = [[c, -q], [conj(q), c]], c =
// cos(theta) (STRANG_XY: cos b cos 2a).  Divided by c a step is
// N = [[1, -tau], [conj(tau), 1]], tau = q / c, and since its diagonal is 1 a
// product W = N_k ... N_1 = [[alpha, -Q], [conj(Q), conj(alpha)]] takes 8
// multiply-adds per step:
//   alpha' = alpha - tau conj(Q),   Q' = Q + tau conj(alpha).
// W differs from U_k ... U_1 by the positive factor 1 / (c_1 ... c_k), and
// det W = |alpha|^2 + |Q|^2 = 1 / (c_1 ... c_k)^2, so the group's operator is
// W / sqrt(det W).  The chain carries Re alpha - 1 (a small part, never rounded
// next to 1), Im alpha and Q:
//   (Re alpha - 1)' = (Re alpha - 1) - (tr Qr + ti Qi)
//   Im alpha'       = Im alpha - (ti Qr - tr Qi)
//   Qr'             = Qr + tr Re alpha + ti Im alpha
//   Qi'             = Qi + ti Re alpha - tr Im alpha
// (Re alpha = 1 + (Re alpha - 1) rounded once per step for the last two).  At
// the end y = det W - 1 = 2 (Re alpha - 1) + (Re alpha - 1)^2 + (Im alpha)^2 +
// |Q|^2 comes from small parts only, f = (1 + y)^(-1/2) - 1 from its binomial
// series, and the compensated update applies
//   M - I = [[am + i ai, -Q'], [conj(Q'), am - i ai]],
//   am = (Re alpha - 1) + f + (Re alpha - 1) f,  ai = Im alpha + f Im alpha,
//   Q' = Q + f Q,
// unitary to the rounding of its small entries.  Per step the chain costs 9
// operations where the product of the U costs 12, and cos(theta) - 1 is never
// evaluated.
//   EXACT:     tau = (tan theta / theta)(dt P_y + i dt P_x) = P + (tan theta/theta - 1) P
//   STRANG_XY: tau = tan b sec 2a + i tan 2a,  b = dt P_y, 2a = dt P_x,
//              tan b sec 2a = tan b + tan b (sec 2a - 1)
// A launch that starts or ends inside a group takes those steps as chains of
// one step each (first, then finish).
// ---------------------------------------------------------------------------

template <typename V>
struct TanChain {
    V as, ai, Qr, Qi;  // Re alpha - 1, Im alpha, Q

    __device__ __forceinline__ void first(V tr, V ti)
    {
        as = vbc<V>(0.0f);
        ai = vbc<V>(0.0f);
        Qr = tr;
        Qi = ti;
    }
    // the second step (alpha = 1 still)
    __device__ __forceinline__ void second(V tr, V ti)
    {
        as = vfma(vneg(tr), Qr, vmul(vneg(ti), Qi));
        ai = vfma(vneg(ti), Qr, vmul(tr, Qi));
        Qr = vadd(Qr, tr);
        Qi = vadd(Qi, ti);
    }
    __device__ __forceinline__ void next(V tr, V ti)
    {
        const V Ar = vadd(as, vbc<V>(1.0f));
        const V nas = vfma(vneg(tr), Qr, vfma(vneg(ti), Qi, as));
        const V nai = vfma(vneg(ti), Qr, vfma(tr, Qi, ai));
        const V nQr = vfma(tr, Ar, vfma(ti, ai, Qr));
        const V nQi = vfma(ti, Ar, vfma(vneg(tr), ai, Qi));
        as = nas;
        ai = nai;
        Qr = nQr;
        Qi = nQi;
    }
    // MAGNUS4 steps, whose N has the diagonal 1 -/+ i tz (see coeffs_tan_magnus):
    //   (Re alpha - 1)' = (Re alpha - 1) + tz Im alpha - (tr Qr + ti Qi)
    //   Im alpha'       = Im alpha - tz Re alpha - (ti Qr - tr Qi)
    //   Qr'             = Qr + tz Qi + tr Re alpha + ti Im alpha
    //   Qi'             = Qi - tz Qr + ti Re alpha - tr Im alpha
    __device__ __forceinline__ void first_z(V tr, V ti, V tz)
    {
        as = vbc<V>(0.0f);
        ai = vneg(tz);
        Qr = tr;
        Qi = ti;
    }
    __device__ __forceinline__ void next_z(V tr, V ti, V tz)
    {
        const V Ar = vadd(as, vbc<V>(1.0f));
        const V nas = vfma(tz, ai, vfma(vneg(tr), Qr, vfma(vneg(ti), Qi, as)));
        const V nai = vfma(vneg(tz), Ar, vfma(vneg(ti), Qr, vfma(tr, Qi, ai)));
        const V nQr = vfma(tz, Qi, vfma(tr, Ar, vfma(ti, ai, Qr)));
        const V nQi = vfma(vneg(tz), Qr, vfma(ti, Ar, vfma(vneg(tr), ai, Qi)));
        as = nas;
        ai = nai;
        Qr = nQr;
        Qi = nQi;
    }
    template <int DF, typename Pt>
    __device__ __forceinline__ void finish(Pt &p) const
    {
        const V y = vfma(as, as, vfma(Qi, Qi, vfma(Qr, Qr, vfma(ai, ai, vadd(as, as)))));
        const V f = vmul(vseries<V, RsqrtCoef, DF, 1>(y), y);
        const V am = vfma(as, f, vadd(as, f));
        apply_group(p, am, vfma(f, ai, ai), vfma(f, Qr, Qr), vfma(f, Qi, Qi));
    }
};

// The coefficient of theta^2 in tan(theta)/theta, rounded to float.  With tan
// degree DT = 1 the EXACT step forms tan(theta)/theta - 1 = c1 theta^2 as
// fma(fl(c1 P_x), P_x, fl(fl(c1 P_y) P_y)): one multiply-add per spinor once the
// column part fl(c1 P_x) and the row part fl(fl(c1 P_y) P_y) are known.
constexpr float kTanC1 = static_cast<float>(kTanSeries[1]);

// tau of one step (contiguous tiles): SCHEME 0 = EXACT, 1 = STRANG_XY.
template <int SCHEME, int DT, typename Pt, typename V>
__device__ __forceinline__ void coeffs_tan(const Pt &p, const float2 &a, V &tr, V &ti)
{
    const V Px = vadd(p.pxh, vadd(vbc<V>(a.x), p.pxl));
    const V Py = vadd(p.pyh, vadd(vbc<V>(a.y), p.pyl));
    if constexpr (SCHEME == 0 && DT == 1) {
        // tan(theta)/theta - 1 = c1 theta^2 = (c1 P_x) P_x + (c1 P_y) P_y, the column
        // and row parts formed apart (the row strips share them)
        const V t1 = vfma(vmul(vbc<V>(kTanC1), Px), Px, vmul(vmul(vbc<V>(kTanC1), Py), Py));
        tr = vfma(t1, Py, Py);
        ti = vfma(t1, Px, Px);
    } else if constexpr (SCHEME == 0) {
        const V x = vfma(Px, Px, vmul(Py, Py));
        const V t1 = vmul(vseries<V, TanCoef, DT, 1>(x), x);  // tan(theta)/theta - 1
        tr = vfma(t1, Py, Py);
        ti = vfma(t1, Px, Px);
    } else {
        const V xx = vmul(Px, Px), xy = vmul(Py, Py);
        const V tb = vfma(vmul(vseries<V, TanCoef, DT, 1>(xy), xy), Py, Py);  // tan b
        ti = vfma(vmul(vseries<V, TanCoef, DT, 1>(xx), xx), Px, Px);          // tan 2a
        const V sc = vmul(vseries<V, SecCoef, DT, 1>(xx), xx);                // sec 2a - 1
        tr = vfma(tb, sc, tb);
    }
}

template <int G, int DT, int SCHEME, typename Pt>
__device__ __forceinline__ void step_group_tan(Pt &p, const float2 *e)
{
    using V = decltype(p.ar);
    TanChain<V> c;
    V tr, ti;
    coeffs_tan<SCHEME, DT>(p, e[0], tr, ti);
    c.first(tr, ti);
    coeffs_tan<SCHEME, DT>(p, e[1], tr, ti);
    c.second(tr, ti);
#pragma unroll kGroupUnroll
    for (int k = 2; k < G; ++k) {
        coeffs_tan<SCHEME, DT>(p, e[k], tr, ti);
        c.next(tr, ti);
    }
    c.template finish<kTanNormDegree(G)>(p);
}

// A step of a grouped run outside whole groups (ragged start or end).
template <int G, int DT, int SCHEME, typename Pt>
__device__ __forceinline__ void step_single_tan(Pt &p, const float2 &e)
{
    using V = decltype(p.ar);
    TanChain<V> c;
    V tr, ti;
    coeffs_tan<SCHEME, DT>(p, e, tr, ti);
    c.first(tr, ti);
    c.template finish<kTanNormDegree(G)>(p);
}

// MAGNUS4 steps in tan-normalised groups (G = 2, 4, 8, 16).  One step is
// exp(-i n.sigma) with n = (dt Pbar, n_z): U = [[c - i qz, -q], [conj(q), c + i
// qz]], c = cos|n|, (q, qz) = sin|n|/|n| (n_y + i n_x, n_z).  Its diagonal is
// complex, but divided by c the step is N = [[1 - i tz, -tau], [conj(tau), 1 + i
// tz]] with (tau, tz) = tan|n|/|n| (n_y + i n_x, n_z), still of the form [[alpha,
// -Q], [conj(Q), conj(alpha)]], so the product W = N_G ... N_1 has that form too
// and det W = prod sec^2 |n_k|: the group's operator is W / sqrt(det W), as for
// EXACT (TanChain::finish).  A chain step (TanChain::next_z) takes 13 operations
// where the product of the U takes 16, and cos|n| - 1 is never evaluated.  The
// tan series is the EXACT one (kTanSeries, degree DT) in x = |n|^2, and tau, tz
// are formed as n + (tan|n|/|n| - 1) n.
template <int DT, typename Pt, typename V>
__device__ __forceinline__ void coeffs_tan_magnus(const Pt &p, const float4 &e, V &tr, V &ti,
                                                  V &tz)
{
    const V Px = vadd(p.pxh, vadd(vbc<V>(e.x), p.pxl));
    const V Py = vadd(p.pyh, vadd(vbc<V>(e.y), p.pyl));
    const V nz = vfma(Px, vbc<V>(e.w), vneg(vmul(Py, vbc<V>(e.z))));
    const V x = vfma(Px, Px, vfma(Py, Py, vmul(nz, nz)));
    const V t1 = vmul(vseries<V, TanCoef, DT, 1>(x), x);  // tan|n|/|n| - 1
    tr = vfma(t1, Py, Py);
    ti = vfma(t1, Px, Px);
    tz = vfma(t1, nz, nz);
}

template <int G, int DT, typename Pt>
__device__ __forceinline__ void step_group_tan_magnus(Pt &p, const float4 *e)
{
    using V = decltype(p.ar);
    TanChain<V> c;
    V tr, ti, tz;
    coeffs_tan_magnus<DT>(p, e[0], tr, ti, tz);
    c.first_z(tr, ti, tz);
#pragma unroll kGroupUnroll
    for (int k = 1; k < G; ++k) {
        coeffs_tan_magnus<DT>(p, e[k], tr, ti, tz);
        c.next_z(tr, ti, tz);
    }
    c.template finish<kTanNormDegree(G)>(p);
}

// A MAGNUS4 step of a grouped run outside whole groups (ragged start or end).
template <int G, int DT, typename Pt>
__device__ __forceinline__ void step_single_tan_magnus(Pt &p, const float4 &e)
{
    using V = decltype(p.ar);
    TanChain<V> c;
    V tr, ti, tz;
    coeffs_tan_magnus<DT>(p, e, tr, ti, tz);
    c.first_z(tr, ti, tz);
    c.template finish<kTanNormDegree(G)>(p);
}

}  // namespace
}  // namespace dsp
