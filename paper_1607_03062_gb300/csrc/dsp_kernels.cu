// dsp_kernels.cu -- sm_103a kernels of the split-operator massless-Dirac solver.
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

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

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
__device__ __forceinline__ float cosm1_f32(float x)
{
    return horner<float, D, 1, 0>(x) * x;
}
template <int D>
__device__ __forceinline__ float sinc_f32(float x)
{
    return horner<float, D, 0, 1>(x);
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

// s + e = a + b exactly (TwoSum, no condition on the magnitudes).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fadd_rn(s, -a);
    e = __fadd_rn(__fadd_rn(a, -__fadd_rn(s, -bb)), __fadd_rn(b, -bb));
}

// The double x as hi + lo floats: hi = x rounded toward zero (same exponent as
// x), lo = the 29 fraction bits hi drops, rounded to a float (x - hi - lo is
// below 2^-48 |x|).  Integer operations only, no FP64 arithmetic.  Values
// below 2^-74 in magnitude keep lo = 0 (their lo is below 2^-97).
__device__ __forceinline__ void split_f64(double x, float &hi, float &lo)
{
    hi = __double2float_rz(x);
    const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned int e = static_cast<unsigned int>(bits >> 52) & 0x7FFu;
    const unsigned int m = static_cast<unsigned int>(bits) & 0x1FFFFFFFu;
    lo = 0.0f;
    if (e >= 949u && e <= 1202u) {  // 2^(e - 1075) is a normal float
        lo = __fmul_rn(__uint2float_rn(m), __int_as_float(static_cast<int>((e - 948u) << 23)));
        if (bits >> 63)
            lo = -lo;
    }
}

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

// |c+|^2 of point idx (global row row0 + idx / nx) as a double: the double-float
// form above, or FP64 for the tiny-|P_out| points.  The spinor is given both
// as hi/lo pairs and (for that FP64 form) as doubles.
struct SpinorDF {
    float arh, arl, aih, ail, brh, brl, bih, bil;
};

__device__ __forceinline__ double project_node(const ReqDesc &R, int64_t col, int64_t row,
                                               const SpinorDF &v, double ar, double ai, double br,
                                               double bi)
{
    const float2 cx = R.nodes_out[col], cy = R.nodes_out[R.nx + row];
    float oh, ol;
    if (project_df(cx.x, cx.y, cy.x, cy.y, v.arh, v.arl, v.aih, v.ail, v.brh, v.brl, v.bih,
                   v.bil, oh, ol))
        return __dadd_rn(static_cast<double>(oh), static_cast<double>(ol));
    const double vs = R.valley > 0 ? 1.0 : -1.0;
    const double px = grid_node(R.px_min, R.hx, col);
    const double py = grid_node(R.py_min, R.hy, R.row0 + row);
    return project_point(px + R.a_out[0], py + R.a_out[1], vs, ar, ai, br, bi);
}

// Fixed pairwise tree over kTilePoints doubles in shared memory (deterministic).
__device__ __forceinline__ double tile_tree_sum(double *red)
{
    for (int s = kTilePoints / 2; s > 0; s >>= 1) {
        for (int t = threadIdx.x; t < s; t += blockDim.x)
            red[t] += red[t + s];
        __syncthreads();
    }
    return red[0];
}

// Locates the request a CTA belongs to (requests are sorted by tile_begin).
__device__ __forceinline__ int find_request(const EvolveArgs &a)
{
    int lo = 0, hi = a.nreq - 1;
    const int b = static_cast<int>(blockIdx.x);
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

// Tuning constants: unroll factors of the step-pair loop and of the chain inside
// a step group (measured fastest fully unrolled, although ptxas then keeps a few
// values in local memory), and spinors per thread of the FP32-mixed kernel (a CTA
// always owns one 1024-point tile).
#ifndef DSP_PAIR_UNROLL
#define DSP_PAIR_UNROLL 2
#endif
#ifndef DSP_MIXED_SPT
#define DSP_MIXED_SPT 4
#endif
#ifndef DSP_MIXED_MINB
#define DSP_MIXED_MINB 2
#endif
#ifndef DSP_PACKED_PAIRS
#define DSP_PACKED_PAIRS 1
#endif
#ifndef DSP_GROUP_UNROLL
#define DSP_GROUP_UNROLL 8
#endif
constexpr int kPairUnroll = DSP_PAIR_UNROLL;
constexpr int kGroupUnroll = DSP_GROUP_UNROLL;  // chain loop inside one group (>= G - 2: whole)
#ifndef DSP_MAGNUS_GROUP_UNROLL
#define DSP_MAGNUS_GROUP_UNROLL 1
#endif
constexpr int kMagnusGroupUnroll = DSP_MAGNUS_GROUP_UNROLL;  // the MAGNUS4 chain's
// Series levels that can run in step groups.  G >= 2 needs theta_max <= 0.1, where a
// level above degree kGroupMaxDegree is chosen only for runs of more than ~3e8 steps;
// the host keeps G = 1 at those levels (choose_group), and no group code is compiled
// for them.
template <int DC, int DS>
constexpr bool kGroupedLevel = DC <= kGroupMaxDegree && DS <= kGroupMaxDegree;
constexpr int kMixedSpt = DSP_MIXED_SPT;
constexpr int kMixedThreads = kTilePoints / kMixedSpt;
constexpr int kMixedMinBlocks = DSP_MIXED_MINB;  // resident CTAs per SM the registers allow
constexpr bool kPackedPairs = DSP_PACKED_PAIRS != 0;  // FP32x2 form of the paired path
constexpr int kF64Threads = kThreads;
static_assert(kTilePoints % kMixedSpt == 0, "a CTA owns one whole tile");

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
template <typename E>
struct Stager {
    unsigned char *smem;
    uint64_t *bars;
    const E *table;  // entry base is element 0 of chunk 0
    int64_t nsteps;
    int nchunks;
    int withhold_first = 0;  // test hook (ReqDesc::withhold_first_copy)
    static constexpr int kCh = kStageBytes / static_cast<int>(sizeof(E));
    static constexpr int kAlign = sizeof(E) >= 16 ? 1 : static_cast<int>(16 / sizeof(E));
    static_assert(16 % sizeof(E) == 0 || sizeof(E) % 16 == 0, "entries tile 16 bytes");
    static_assert(kCh % kAlign == 0, "chunks start on 16-byte boundaries");

    __device__ __forceinline__ const E *stage(int c) const
    {
        return reinterpret_cast<const E *>(smem + (c & 1) * kStageBytes);
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
        bulk_load(smem + (c & 1) * kStageBytes, table + static_cast<int64_t>(c) * kCh, bytes,
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
// FP32_MIXED step
// ---------------------------------------------------------------------------

struct MixedPoint {
    float ar, ai, br, bi;      // hi parts of psi = (a, b)
    float lar, lai, lbr, lbi;  // lo parts
    float pxh, pxl, pyh, pyl;  // dt * p as hi + lo
};

// Coefficients of U - I = [[cm1 - i qz, -q], [conj(q), cm1 + i qz]], q = qr + i qi,
// for the step with kinematic momentum dt*P = (Px, Py).  EXACT and STRANG_XY have
// qz = 0.
template <int SCHEME, int DC, int DS>
__device__ __forceinline__ void step_coeffs_f32(float Px, float Py, float2 d, float &cm1,
                                                float &qr, float &qi, float &qz)
{
    if constexpr (SCHEME == 0) {
        const float x = fmaf(Px, Px, Py * Py);  // theta^2
        cm1 = cosm1_f32<DC>(x);
        const float sn = sinc_f32<DS>(x);
        qr = sn * Py;
        qi = sn * Px;
        qz = 0.0f;
    } else if constexpr (SCHEME == 1) {
        // e^{-i a sx} e^{-i b sy} e^{-i a sx}, a = dt Px / 2, b = dt Py:
        //   = [[cos b cos 2a, -(sin b + i cos b sin 2a)], [sin b - i cos b sin 2a, cos b cos 2a]]
        const float xx = Px * Px, xy = Py * Py;
        const float cmx = cosm1_f32<DC>(xx), cmy = cosm1_f32<DC>(xy);
        const float sx = Px * sinc_f32<DS>(xx);
        cm1 = fmaf(cmx, cmy, cmx) + cmy;
        qr = Py * sinc_f32<DS>(xy);
        qi = fmaf(cmy, sx, sx);
        qz = 0.0f;
    } else {
        // MAGNUS4: exp(-i n.sigma), n = (dt Pbar, n_z), n_z = -(sqrt 3/6) (dt P1 x dt P2)_z
        // = (dt Pbar x D')_z with D' = -(sqrt 3/6) dt (A2 - A1) from the table (the
        // cross product of the two nearly parallel momenta is never formed).
        const float nz = fmaf(Px, d.y, -(Py * d.x));
        const float x = fmaf(Px, Px, fmaf(Py, Py, nz * nz));
        cm1 = cosm1_f32<DC>(x);
        const float sn = sinc_f32<DS>(x);
        qr = sn * Py;
        qi = sn * Px;
        qz = sn * nz;
    }
}

// psi <- U psi as psi_hi + (U - I) psi_hi + psi_lo, the rounding error of the
// hi update carried into lo (Fast2Sum).
template <int SCHEME>
__device__ __forceinline__ void apply_f32(MixedPoint &s, float cm1, float qr, float qi, float qz)
{
    float dar, dai, dbr, dbi;
    if constexpr (SCHEME == 2) {
        dar = fmaf(cm1, s.ar, fmaf(qz, s.ai, fmaf(-qr, s.br, fmaf(qi, s.bi, s.lar))));
        dai = fmaf(cm1, s.ai, fmaf(-qz, s.ar, fmaf(-qr, s.bi, fmaf(-qi, s.br, s.lai))));
        dbr = fmaf(cm1, s.br, fmaf(-qz, s.bi, fmaf(qr, s.ar, fmaf(qi, s.ai, s.lbr))));
        dbi = fmaf(cm1, s.bi, fmaf(qz, s.br, fmaf(qr, s.ai, fmaf(-qi, s.ar, s.lbi))));
    } else {
        dar = fmaf(cm1, s.ar, fmaf(-qr, s.br, fmaf(qi, s.bi, s.lar)));
        dai = fmaf(cm1, s.ai, fmaf(-qr, s.bi, fmaf(-qi, s.br, s.lai)));
        dbr = fmaf(cm1, s.br, fmaf(qr, s.ar, fmaf(qi, s.ai, s.lbr)));
        dbi = fmaf(cm1, s.bi, fmaf(qr, s.ai, fmaf(-qi, s.ar, s.lbi)));
    }
    float t;
    t = s.ar + dar; s.lar = dar - (t - s.ar); s.ar = t;
    t = s.ai + dai; s.lai = dai - (t - s.ai); s.ai = t;
    t = s.br + dbr; s.lbr = dbr - (t - s.br); s.br = t;
    t = s.bi + dbi; s.lbi = dbi - (t - s.bi); s.bi = t;
}

// dt*P = dt p_hi + (dt A + dt p_lo), rounded in that order.
[[maybe_unused]] __device__ __forceinline__ float momentum_f32(float ph, float a, float pl)
{
    return __fadd_rn(ph, __fadd_rn(a, pl));
}

template <int SCHEME, int DC, int DS>
__device__ __forceinline__ void step_mixed(MixedPoint &p, const float2 &a, float2 d)
{
    float cm1, qr, qi, qz;
    step_coeffs_f32<SCHEME, DC, DS>(momentum_f32(p.pxh, a.x, p.pxl),
                                    momentum_f32(p.pyh, a.y, p.pyl), d, cm1, qr, qi, qz);
    apply_f32<SCHEME>(p, cm1, qr, qi, qz);
}

// Two EXACT steps at once: with U_k = I + [[m_k, -q_k], [conj(q_k), m_k]],
//   U_2 U_1 - I = [[al - 1, -Q], [conj(Q), conj(al) - 1]],
//   al - 1 = m1 + m2 + m1 m2 - q2 conj(q1),  Q = q1 + q2 + m2 q1 + m1 q2,
// applied with one compensated update (the product of two SU(2) steps is SU(2)).
template <int DC, int DS>
__device__ __forceinline__ void step_pair_mixed(MixedPoint &p, const float2 &a0, const float2 &a1)
{
    float m1, q1r, q1i, m2, q2r, q2i, z;
    step_coeffs_f32<0, DC, DS>(momentum_f32(p.pxh, a0.x, p.pxl), momentum_f32(p.pyh, a0.y, p.pyl),
                               make_float2(0.0f, 0.0f), m1, q1r, q1i, z);
    step_coeffs_f32<0, DC, DS>(momentum_f32(p.pxh, a1.x, p.pxl), momentum_f32(p.pyh, a1.y, p.pyl),
                               make_float2(0.0f, 0.0f), m2, q2r, q2i, z);
    const float alm1 = fmaf(m1, m2, m1 + m2) - fmaf(q2r, q1r, q2i * q1i);
    const float ali = fmaf(q2r, q1i, -(q2i * q1r));
    const float Qr = fmaf(m2, q1r, q1r) + fmaf(m1, q2r, q2r);
    const float Qi = fmaf(m2, q1i, q1i) + fmaf(m1, q2i, q2i);
    const float dar = fmaf(alm1, p.ar, fmaf(-ali, p.ai, fmaf(-Qr, p.br, fmaf(Qi, p.bi, p.lar))));
    const float dai = fmaf(alm1, p.ai, fmaf(ali, p.ar, fmaf(-Qr, p.bi, fmaf(-Qi, p.br, p.lai))));
    const float dbr = fmaf(alm1, p.br, fmaf(ali, p.bi, fmaf(Qr, p.ar, fmaf(Qi, p.ai, p.lbr))));
    const float dbi = fmaf(alm1, p.bi, fmaf(-ali, p.br, fmaf(Qr, p.ai, fmaf(-Qi, p.ar, p.lbi))));
    float t;
    t = p.ar + dar; p.lar = dar - (t - p.ar); p.ar = t;
    t = p.ai + dai; p.lai = dai - (t - p.ai); p.ai = t;
    t = p.br + dbr; p.lbr = dbr - (t - p.br); p.br = t;
    t = p.bi + dbi; p.lbi = dbi - (t - p.bi); p.bi = t;
}

// ---------------------------------------------------------------------------
// Packed FP32x2 form of the paired EXACT path: lane 0 and lane 1 of every
// float2 belong to two different momenta, and every operation is the scalar
// path's operation, in the same order, so each lane's result is bitwise the
// scalar result (the packed instructions round each lane like the scalar ones).
// One instruction then issues the arithmetic of two spinors.
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

// One EXACT step (apply_f32<0> with cm1 = m, q = (qr, qi)).
template <int DC, int DS>
__device__ __forceinline__ void step_exact2(MixedPack &p, const float2 &a)
{
    float2 m, qr, qi;
    coeffs_exact2<DC, DS>(p, a, m, qr, qi);
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

// Two EXACT steps multiplied, then one update (step_pair_mixed on two momenta).
template <int DC, int DS>
__device__ __forceinline__ void step_pair2(MixedPack &p, const float2 &a0, const float2 &a1)
{
    float2 m1, q1r, q1i, m2, q2r, q2i;
    coeffs_exact2<DC, DS>(p, a0, m1, q1r, q1i);
    coeffs_exact2<DC, DS>(p, a1, m2, q2r, q2i);
    const float2 alm1 = sub2(fma2(m1, m2, add2(m1, m2)), fma2(q2r, q1r, mul2(q2i, q1i)));
    const float2 ali = fma2(q2r, q1i, neg2(mul2(q2i, q1r)));
    const float2 Qr = add2(fma2(m2, q1r, q1r), fma2(m1, q2r, q2r));
    const float2 Qi = add2(fma2(m2, q1i, q1i), fma2(m1, q2i, q2i));
    apply2(p, alm1, ali, Qr, Qi);
}

// ---------------------------------------------------------------------------
// Groups of G EXACT steps (G = 4, 8), written once for one momentum (V = float,
// MixedPoint) and for two (V = float2, MixedPack) with non-contracting
// intrinsics, so both forms perform the same roundings.
//
// The product U_k ... U_1 = [[alpha, -Q], [conj(Q), conj(alpha)]] is carried as
// (Re alpha, Im alpha, Q).  With U_k = [[1 + m, -q], [conj(q), 1 + m]],
// m = cos(theta_k) - 1, q = sin(theta_k)/theta_k (dt P_y + i dt P_x):
//   alpha' = alpha + m alpha - q conj(Q),   Q' = Q + m Q + q conj(alpha).
// No coefficient of the form 1 + (small) is ever rounded: cos(theta) enters as
// X + m X and sin(theta)/theta as P + (sinc - 1) P, both accurate to the
// rounding of the small part.  (Rounding cos(theta) itself to FP32 next to 1
// errs by up to 3e-8 absolute, the same for every step while theta barely
// changes, and the step angle then carries a relative bias of that size, which
// grows along the whole evolution.)  Re alpha is held near 1, where FP32
// resolves it only to ~6e-8; Re alpha - 1 is rebuilt at the end of the group
// from the other three entries and unitarity, (1 + am)^2 + ai^2 + |Q|^2 = 1, by
// one Newton step, so the operator applied is unitary to the rounding of its
// entries.
// ---------------------------------------------------------------------------

// Either set of forms can go unused, depending on the build (the float forms serve
// builds without the packed path: DSP_PACKED_PAIRS=0 or an odd DSP_MIXED_SPT).
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

// m = cos(theta) - 1 and q = (qr, qi) of one EXACT step at dt P = dt p + table
// entry a, with q = P + (sinc - 1) P.
template <int DC, int DS, typename Pt, typename V>
__device__ __forceinline__ void coeffs_group(const Pt &p, const float2 &a, V &m, V &qr, V &qi)
{
    const V Px = vadd(p.pxh, vadd(vbc<V>(a.x), p.pxl));
    const V Py = vadd(p.pyh, vadd(vbc<V>(a.y), p.pyl));
    const V x = vfma(Px, Px, vmul(Py, Py));
    m = vmul(vhorner<V, DC, 1, 0>(x), x);
    const V s1 = vmul(vhorner<V, DS, 1, 1>(x), x);  // sin(theta)/theta - 1
    qr = vfma(s1, Py, Py);
    qi = vfma(s1, Px, Px);
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
// sin b likewise, cos b sin 2a = sin 2a + cy sin 2a.
template <int DC, int DS, typename Pt, typename V>
__device__ __forceinline__ void coeffs_strang_group(const Pt &p, const float2 &a, V &m, V &qr,
                                                    V &qi)
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

// (m, q) of one step of an EXACT-structured scheme: 0 = EXACT, 1 = STRANG_XY.
template <int SCHEME, int DC, int DS, typename Pt, typename V>
__device__ __forceinline__ void coeffs_scheme(const Pt &p, const float2 &a, V &m, V &qr, V &qi)
{
    if constexpr (SCHEME == 1)
        coeffs_strang_group<DC, DS>(p, a, m, qr, qi);
    else
        coeffs_group<DC, DS>(p, a, m, qr, qi);
}

// One step alone through the group update (ragged ends of a grouped STRANG_XY
// run, or all of an ungrouped one): U - I = [[m, -q], [conj(q), m]].
template <int SCHEME, int DC, int DS, typename Pt>
__device__ __forceinline__ void step_single_scheme(Pt &p, const float2 &a)
{
    using V = decltype(p.ar);
    V m, qr, qi;
    coeffs_scheme<SCHEME, DC, DS>(p, a, m, qr, qi);
    apply_group(p, m, vbc<V>(0.0f), qr, qi);
}

// The chain, one step k >= 2 at a time (the second step, with Im alpha still 0,
// drops its terms):
//   Re alpha' = Re alpha + m Re alpha - (qr Qr + qi Qi)
//   Im alpha' = Im alpha + m Im alpha - (qi Qr - qr Qi)
//   Qr'       = Qr + m Qr + qr Re alpha + qi Im alpha
//   Qi'       = Qi + m Qi + qi Re alpha - qr Im alpha
template <int G, int DC, int DS, int SCHEME = 0, typename Pt>
__device__ __forceinline__ void step_group(Pt &p, const float2 *e)
{
    using V = decltype(p.ar);
    V m, qr, qi, Qr, Qi;
    coeffs_scheme<SCHEME, DC, DS>(p, e[0], m, Qr, Qi);
    V Ar = vadd(m, vbc<V>(1.0f));
    coeffs_scheme<SCHEME, DC, DS>(p, e[1], m, qr, qi);
    V ai = vfma(vneg(qi), Qr, vmul(qr, Qi));
    V nAr = vfma(m, Ar, vfma(vneg(qr), Qr, vfma(vneg(qi), Qi, Ar)));
    V nQr = vfma(m, Qr, vfma(qr, Ar, Qr));
    V nQi = vfma(m, Qi, vfma(qi, Ar, Qi));
    Ar = nAr;
    Qr = nQr;
    Qi = nQi;
#pragma unroll kGroupUnroll
    for (int k = 2; k < G; ++k) {
        coeffs_scheme<SCHEME, DC, DS>(p, e[k], m, qr, qi);
        nAr = vfma(m, Ar, vfma(vneg(qr), Qr, vfma(vneg(qi), Qi, Ar)));
        const V nai = vfma(m, ai, vfma(vneg(qi), Qr, vfma(qr, Qi, ai)));
        nQr = vfma(m, Qr, vfma(qr, Ar, vfma(qi, ai, Qr)));
        nQi = vfma(m, Qi, vfma(qi, Ar, vfma(vneg(qr), ai, Qi)));
        Ar = nAr;
        ai = nai;
        Qr = nQr;
        Qi = nQi;
    }
    V am = vadd(Ar, vbc<V>(-1.0f));  // exact: Re alpha is within [1/2, 2]
    const V u = vfma(am, am, vfma(Qi, Qi, vfma(Qr, Qr, vfma(ai, ai, vadd(am, am)))));
    am = vfma(vneg(u), vfma(vbc<V>(-0.5f), am, vbc<V>(0.5f)), am);  // am -= u / (2 (1 + am))
    apply_group(p, am, ai, Qr, Qi);
}

// MAGNUS4 steps in groups (G = 2, 4, 8).  One step is exp(-i n.sigma) with
// n = (dt Pbar, n_z): U = [[1 + m - i qz, -q], [conj(q), 1 + m + i qz]], m =
// cos|n| - 1, (q, qz) = sin|n|/|n| (n_y + i n_x, n_z), formed as n + (sinc - 1) n.
// The chain is the EXACT one with the sigma_z terms added:
//   Re alpha' = Re alpha + m Re alpha + qz Im alpha - (qr Qr + qi Qi)
//   Im alpha' = Im alpha + m Im alpha - qz Re alpha - (qi Qr - qr Qi)
//   Qr'       = Qr + m Qr + qz Qi + qr Re alpha + qi Im alpha
//   Qi'       = Qi + m Qi - qz Qr + qi Re alpha - qr Im alpha
// starting from alpha = 1 + m - i qz, Q = q of the group's first step, then the
// same unitarity rebuild of Re alpha - 1 and compensated update as EXACT groups.
template <int DC, int DS, typename Pt, typename V>
__device__ __forceinline__ void coeffs_magnus_group(const Pt &p, const float4 &e, V &m, V &qr,
                                                    V &qi, V &qz)
{
    const V Px = vadd(p.pxh, vadd(vbc<V>(e.x), p.pxl));
    const V Py = vadd(p.pyh, vadd(vbc<V>(e.y), p.pyl));
    const V nz = vfma(Px, vbc<V>(e.w), vneg(vmul(Py, vbc<V>(e.z))));
    const V x = vfma(Px, Px, vfma(Py, Py, vmul(nz, nz)));
    m = vmul(vhorner<V, DC, 1, 0>(x), x);
    const V s1 = vmul(vhorner<V, DS, 1, 1>(x), x);  // sin|n|/|n| - 1
    qr = vfma(s1, Py, Py);
    qi = vfma(s1, Px, Px);
    qz = vfma(s1, nz, nz);
}

template <int G, int DC, int DS, typename Pt>
__device__ __forceinline__ void step_group_magnus(Pt &p, const float4 *e)
{
    using V = decltype(p.ar);
    V m, qr, qi, qz, Qr, Qi;
    coeffs_magnus_group<DC, DS>(p, e[0], m, Qr, Qi, qz);
    V Ar = vadd(m, vbc<V>(1.0f));
    V ai = vneg(qz);
#pragma unroll kMagnusGroupUnroll
    for (int k = 1; k < G; ++k) {
        coeffs_magnus_group<DC, DS>(p, e[k], m, qr, qi, qz);
        const V nAr = vfma(m, Ar, vfma(qz, ai, vfma(vneg(qr), Qr, vfma(vneg(qi), Qi, Ar))));
        const V nai = vfma(m, ai, vfma(vneg(qz), Ar, vfma(vneg(qi), Qr, vfma(qr, Qi, ai))));
        const V nQr = vfma(m, Qr, vfma(qz, Qi, vfma(qr, Ar, vfma(qi, ai, Qr))));
        const V nQi = vfma(m, Qi, vfma(vneg(qz), Qr, vfma(qi, Ar, vfma(vneg(qr), ai, Qi))));
        Ar = nAr;
        ai = nai;
        Qr = nQr;
        Qi = nQi;
    }
    V am = vadd(Ar, vbc<V>(-1.0f));  // exact: Re alpha is within [1/2, 2]
    const V u = vfma(am, am, vfma(Qi, Qi, vfma(Qr, Qr, vfma(ai, ai, vadd(am, am)))));
    am = vfma(vneg(u), vfma(vbc<V>(-0.5f), am, vbc<V>(0.5f)), am);  // am -= u / (2 (1 + am))
    apply_group(p, am, ai, Qr, Qi);
}

template <int SCHEME, int DC, int DS>
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

    constexpr bool packed = kPackedPairs && S % 2 == 0;
    MixedPack pk[packed ? S / 2 : 1];
    if constexpr (packed) {  // FP32x2: spinors (2k, 2k + 1) share each instruction
#pragma unroll
        for (int k = 0; k < S / 2; ++k)
            pk[k] = pack_points(pt[2 * k], pt[2 * k + 1]);
    }
    bool ok;
    if constexpr (SCHEME == 0 && packed) {
        const auto single = [&](const float2 &e) {
#pragma unroll
            for (int k = 0; k < S / 2; ++k)
                step_exact2<DC, DS>(pk[k], e);
        };
        if constexpr (kGroupedLevel<DC, DS>) {
            if (R.group == kGroupMax) {
                ok = run_step_groups<float2, kGroupMax>(R, smem, bars, err, single,
                                                        [&](const float2 *e) {
#pragma unroll
                    for (int k = 0; k < S / 2; ++k)
                        step_group<kGroupMax, DC, DS>(pk[k], e);
                });
            } else if (R.group == 8) {
                ok = run_step_groups<float2, 8>(R, smem, bars, err, single, [&](const float2 *e) {
#pragma unroll
                    for (int k = 0; k < S / 2; ++k)
                        step_group<8, DC, DS>(pk[k], e);
                });
            } else if (R.group == 4) {
                ok = run_step_groups<float2, 4>(R, smem, bars, err, single, [&](const float2 *e) {
#pragma unroll
                    for (int k = 0; k < S / 2; ++k)
                        step_group<4, DC, DS>(pk[k], e);
                });
            } else if (R.group == 2) {
                ok = run_step_groups<float2, 2>(R, smem, bars, err, single, [&](const float2 *e) {
#pragma unroll
                    for (int k = 0; k < S / 2; ++k)
                        step_pair2<DC, DS>(pk[k], e[0], e[1]);
                });
            } else {
                ok = run_steps<float2>(R, smem, bars, err, single);
            }
        } else {  // no group paths at this level (the host keeps G = 1)
            ok = run_steps<float2>(R, smem, bars, err, single);
        }
    } else if constexpr (SCHEME == 1 && packed) {
        const auto single = [&](const float2 &e) {
#pragma unroll
            for (int k = 0; k < S / 2; ++k)
                step_single_scheme<1, DC, DS>(pk[k], e);
        };
        if constexpr (kGroupedLevel<DC, DS>) {
            if (R.group == 8) {
                ok = run_step_groups<float2, 8>(R, smem, bars, err, single, [&](const float2 *e) {
#pragma unroll
                    for (int k = 0; k < S / 2; ++k)
                        step_group<8, DC, DS, 1>(pk[k], e);
                });
            } else if (R.group == 4) {
                ok = run_step_groups<float2, 4>(R, smem, bars, err, single, [&](const float2 *e) {
#pragma unroll
                    for (int k = 0; k < S / 2; ++k)
                        step_group<4, DC, DS, 1>(pk[k], e);
                });
            } else if (R.group == 2) {
                ok = run_step_groups<float2, 2>(R, smem, bars, err, single, [&](const float2 *e) {
#pragma unroll
                    for (int k = 0; k < S / 2; ++k)
                        step_group<2, DC, DS, 1>(pk[k], e);
                });
            } else {
                ok = run_steps<float2>(R, smem, bars, err, single);
            }
        } else {  // no group paths at this level (the host keeps G = 1)
            ok = run_steps<float2>(R, smem, bars, err, single);
        }
    } else if constexpr (SCHEME == 2 && packed) {
        const auto single = [&](const float4 &e) {
#pragma unroll
            for (int k = 0; k < S / 2; ++k)
                step_magnus2<DC, DS>(pk[k], e);
        };
        if constexpr (kGroupedLevel<DC, DS>) {
            if (R.group == 8) {
                ok = run_step_groups<float4, 8>(R, smem, bars, err, single, [&](const float4 *e) {
#pragma unroll
                    for (int k = 0; k < S / 2; ++k)
                        step_group_magnus<8, DC, DS>(pk[k], e);
                });
            } else if (R.group == 4) {
                ok = run_step_groups<float4, 4>(R, smem, bars, err, single, [&](const float4 *e) {
#pragma unroll
                    for (int k = 0; k < S / 2; ++k)
                        step_group_magnus<4, DC, DS>(pk[k], e);
                });
            } else if (R.group == 2) {
                ok = run_step_groups<float4, 2>(R, smem, bars, err, single, [&](const float4 *e) {
#pragma unroll
                    for (int k = 0; k < S / 2; ++k)
                        step_group_magnus<2, DC, DS>(pk[k], e);
                });
            } else {
                ok = run_steps<float4>(R, smem, bars, err, single);
            }
        } else {  // no group paths at this level (the host keeps G = 1)
            ok = run_steps<float4>(R, smem, bars, err, single);
        }
    } else if constexpr (SCHEME == 0) {
        const auto single = [&](const float2 &e) {
#pragma unroll
            for (int s = 0; s < S; ++s)
                step_mixed<SCHEME, DC, DS>(pt[s], e, make_float2(0.0f, 0.0f));
        };
        if constexpr (kGroupedLevel<DC, DS>) {
            if (R.group == kGroupMax) {
                ok = run_step_groups<float2, kGroupMax>(R, smem, bars, err, single,
                                                        [&](const float2 *e) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        step_group<kGroupMax, DC, DS>(pt[s], e);
                });
            } else if (R.group == 8) {
                ok = run_step_groups<float2, 8>(R, smem, bars, err, single, [&](const float2 *e) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        step_group<8, DC, DS>(pt[s], e);
                });
            } else if (R.group == 4) {
                ok = run_step_groups<float2, 4>(R, smem, bars, err, single, [&](const float2 *e) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        step_group<4, DC, DS>(pt[s], e);
                });
            } else if (R.group == 2) {
                ok = run_step_groups<float2, 2>(R, smem, bars, err, single, [&](const float2 *e) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        step_pair_mixed<DC, DS>(pt[s], e[0], e[1]);
                });
            } else {
                ok = run_steps<float2>(R, smem, bars, err, single);
            }
        } else {  // no group paths at this level (the host keeps G = 1)
            ok = run_steps<float2>(R, smem, bars, err, single);
        }
    } else if constexpr (SCHEME == 2) {
        const auto single = [&](const float4 &e) {
#pragma unroll
            for (int s = 0; s < S; ++s)
                step_mixed<SCHEME, DC, DS>(pt[s], make_float2(e.x, e.y), make_float2(e.z, e.w));
        };
        if constexpr (kGroupedLevel<DC, DS>) {
            if (R.group == 8) {
                ok = run_step_groups<float4, 8>(R, smem, bars, err, single, [&](const float4 *e) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        step_group_magnus<8, DC, DS>(pt[s], e);
                });
            } else if (R.group == 4) {
                ok = run_step_groups<float4, 4>(R, smem, bars, err, single, [&](const float4 *e) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        step_group_magnus<4, DC, DS>(pt[s], e);
                });
            } else if (R.group == 2) {
                ok = run_step_groups<float4, 2>(R, smem, bars, err, single, [&](const float4 *e) {
#pragma unroll
                    for (int s = 0; s < S; ++s)
                        step_group_magnus<2, DC, DS>(pt[s], e);
                });
            } else {
                ok = run_steps<float4>(R, smem, bars, err, single);
            }
        } else {  // no group paths at this level (the host keeps G = 1)
            ok = run_steps<float4>(R, smem, bars, err, single);
        }
    } else {
        ok = run_steps<float2>(R, smem, bars, err, [&](const float2 &e) {
#pragma unroll
            for (int s = 0; s < S; ++s)
                step_mixed<SCHEME, DC, DS>(pt[s], e, make_float2(0.0f, 0.0f));
        });
    }
    if constexpr (packed) {
#pragma unroll
        for (int k = 0; k < S / 2; ++k)
            unpack_points(pk[k], pt[2 * k], pt[2 * k + 1]);
    }
    if (!ok)
        return;

    double cp2[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t idx = base + s * kMixedThreads + tid;
        cp2[s] = 0.0;
        if (idx < R.n_points) {
            if (R.store_state) {
                hi_plane[idx] = make_float4(pt[s].ar, pt[s].ai, pt[s].br, pt[s].bi);
                lo_plane[idx] = make_float4(pt[s].lar, pt[s].lai, pt[s].lbr, pt[s].lbi);
            }
            if (R.project) {
                const SpinorDF v{pt[s].ar, pt[s].lar, pt[s].ai, pt[s].lai,
                                 pt[s].br, pt[s].lbr, pt[s].bi, pt[s].lbi};
                cp2[s] = project_node(R, idx % R.nx, idx / R.nx, v,
                                      static_cast<double>(pt[s].ar) + pt[s].lar,
                                      static_cast<double>(pt[s].ai) + pt[s].lai,
                                      static_cast<double>(pt[s].br) + pt[s].lbr,
                                      static_cast<double>(pt[s].bi) + pt[s].lbi);
                if (R.map)
                    static_cast<float *>(R.map)[idx] = static_cast<float>(cp2[s]);
            }
        }
    }
    if (R.project) {
        double *red = reinterpret_cast<double *>(smem);  // the table stages are free now
#pragma unroll
        for (int s = 0; s < S; ++s)
            red[s * kMixedThreads + tid] = cp2[s];
        __syncthreads();
        const double sum = tile_tree_sum(red);
        if (tid == 0)
            R.partials[tile] = sum;
    }
}

// ---------------------------------------------------------------------------
// FP64 step
// ---------------------------------------------------------------------------

struct F64Point {
    double ar, ai, br, bi;
    double tx, ty;  // dt * p (times the valley sign)
};

template <int SCHEME, int DC, int DS>
__device__ __forceinline__ void step_f64(F64Point &s, double2 a, double2 d)
{
    const double Px = s.tx + a.x, Py = s.ty + a.y;  // dt * P (times the valley sign)
    double c, qr, qi, qz = 0.0;
    if constexpr (SCHEME == 0) {
        const double x = fma(Px, Px, Py * Py);
        c = cos_f64<DC>(x);
        const double sn = sinc_f64<DS>(x);
        qr = sn * Py;
        qi = sn * Px;
    } else if constexpr (SCHEME == 1) {
        const double xx = Px * Px, xy = Py * Py;
        const double cy = cos_f64<DC>(xy);
        c = cy * cos_f64<DC>(xx);
        qr = Py * sinc_f64<DS>(xy);
        qi = cy * (Px * sinc_f64<DS>(xx));
    } else {
        const double nz = fma(Px, d.y, -(Py * d.x));  // see step_coeffs_f32
        const double x = fma(Px, Px, fma(Py, Py, nz * nz));
        c = cos_f64<DC>(x);
        const double sn = sinc_f64<DS>(x);
        qr = sn * Py;
        qi = sn * Px;
        qz = sn * nz;
    }
    // a' = (c - i qz) a - q b ; b' = conj(q) a + (c + i qz) b, q = qr + i qi
    double nar, nai, nbr, nbi;
    if constexpr (SCHEME == 2) {
        nar = fma(c, s.ar, fma(qz, s.ai, fma(-qr, s.br, qi * s.bi)));
        nai = fma(c, s.ai, fma(-qz, s.ar, fma(-qr, s.bi, -(qi * s.br))));
        nbr = fma(c, s.br, fma(-qz, s.bi, fma(qr, s.ar, qi * s.ai)));
        nbi = fma(c, s.bi, fma(qz, s.br, fma(qr, s.ai, -(qi * s.ar))));
    } else {
        nar = fma(c, s.ar, fma(-qr, s.br, qi * s.bi));
        nai = fma(c, s.ai, fma(-qr, s.bi, -(qi * s.br)));
        nbr = fma(c, s.br, fma(qr, s.ar, qi * s.ai));
        nbi = fma(c, s.bi, fma(qr, s.ai, -(qi * s.ar)));
    }
    s.ar = nar; s.ai = nai; s.br = nbr; s.bi = nbi;
}

template <int SCHEME, int DC, int DS>
__device__ void body_f64(const ReqDesc &R, int tile, unsigned char *smem, uint64_t *bars, int *err)
{
    constexpr int S = kSpinorsPerThread;
    const int tid = threadIdx.x;
    const int64_t base = static_cast<int64_t>(tile) * kTilePoints;
    const double vs = R.valley > 0 ? 1.0 : -1.0;
    double2 *a_plane = static_cast<double2 *>(R.state);
    double2 *b_plane = a_plane + R.n_points;

    F64Point pt[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t idx = base + s * kThreads + tid;
        const bool valid = idx < R.n_points;
        double px = 0.0, py = 0.0;
        if (valid) {
            px = grid_node(R.px_min, R.hx, idx % R.nx);
            py = grid_node(R.py_min, R.hy, R.row0 + idx / R.nx);
        }
        pt[s].tx = vs * (R.dt * px);  // valley K- is stepped as K+ on -P
        pt[s].ty = vs * (R.dt * py);
        if (R.fresh || !valid) {
            if (R.init_identity) {
                pt[s].ar = 1.0; pt[s].ai = 0.0; pt[s].br = 0.0; pt[s].bi = 0.0;
            } else {
                initial_spinor(px + R.a_in[0], py + R.a_in[1], vs, pt[s].ar, pt[s].ai, pt[s].br,
                               pt[s].bi);
            }
        } else {
            const double2 a = a_plane[idx], b = b_plane[idx];
            pt[s].ar = a.x; pt[s].ai = a.y; pt[s].br = b.x; pt[s].bi = b.y;
        }
    }

    bool ok;
    if constexpr (SCHEME == 2) {
        ok = run_steps<F64G2>(R, smem, bars, err, [&](const F64G2 &e) {
#pragma unroll
            for (int s = 0; s < S; ++s)
                step_f64<SCHEME, DC, DS>(pt[s], e.a, e.d);
        });
    } else {
        ok = run_steps<double2>(R, smem, bars, err, [&](const double2 &e) {
#pragma unroll
            for (int s = 0; s < S; ++s)
                step_f64<SCHEME, DC, DS>(pt[s], e, make_double2(0.0, 0.0));
        });
    }
    if (!ok)
        return;

    double cp2[S];
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t idx = base + s * kThreads + tid;
        cp2[s] = 0.0;
        if (idx < R.n_points) {
            if (R.store_state) {
                a_plane[idx] = make_double2(pt[s].ar, pt[s].ai);
                b_plane[idx] = make_double2(pt[s].br, pt[s].bi);
            }
            if (R.project) {
                SpinorDF v;
                split_f64(pt[s].ar, v.arh, v.arl);
                split_f64(pt[s].ai, v.aih, v.ail);
                split_f64(pt[s].br, v.brh, v.brl);
                split_f64(pt[s].bi, v.bih, v.bil);
                cp2[s] = project_node(R, idx % R.nx, idx / R.nx, v, pt[s].ar, pt[s].ai, pt[s].br,
                                      pt[s].bi);
                if (R.map)
                    static_cast<double *>(R.map)[idx] = cp2[s];
            }
        }
    }
    if (R.project) {
        double *red = reinterpret_cast<double *>(smem);
#pragma unroll
        for (int s = 0; s < S; ++s)
            red[s * kThreads + tid] = cp2[s];
        __syncthreads();
        const double sum = tile_tree_sum(red);
        if (tid == 0)
            R.partials[tile] = sum;
    }
}

// Block-uniform dispatch on the request's series level (compile-time degrees).
template <int SCHEME, int L>
__device__ __forceinline__ void dispatch_mixed(const ReqDesc &R, int tile, unsigned char *smem,
                                               uint64_t *bars, int *err)
{
    if (R.level == L || L + 1 == kNumLevels)
        body_mixed<SCHEME, kLevelsF32[L].dc, kLevelsF32[L].ds>(R, tile, smem, bars, err);
    else if constexpr (L + 1 < kNumLevels)
        dispatch_mixed<SCHEME, L + 1>(R, tile, smem, bars, err);
}

template <int SCHEME, int L>
__device__ __forceinline__ void dispatch_f64(const ReqDesc &R, int tile, unsigned char *smem,
                                             uint64_t *bars, int *err)
{
    if (R.level == L || L + 1 == kNumLevels)
        body_f64<SCHEME, kLevelsF64[L].dc, kLevelsF64[L].ds>(R, tile, smem, bars, err);
    else if constexpr (L + 1 < kNumLevels)
        dispatch_f64<SCHEME, L + 1>(R, tile, smem, bars, err);
}

// ---------------------------------------------------------------------------
// Kernels
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
        dispatch_mixed<0, 0>(R, tile, smem, bars, R.err);
    else if (R.scheme == 1)
        dispatch_mixed<1, 0>(R, tile, smem, bars, R.err);
    else
        dispatch_mixed<2, 0>(R, tile, smem, bars, R.err);
}

__global__ void __launch_bounds__(kThreads, 1)
    evolve_f64_kernel(const __grid_constant__ EvolveArgs args)
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
        dispatch_f64<0, 0>(R, tile, smem, bars, R.err);
    else if (R.scheme == 1)
        dispatch_f64<1, 0>(R, tile, smem, bars, R.err);
    else
        dispatch_f64<2, 0>(R, tile, smem, bars, R.err);
}

// Projection of a state already on the device (a launch with no steps): one CTA
// per 1024-point tile, kProjThreads threads x kProjPoints points, loads of the
// whole tile issued before any arithmetic.  The value of each point comes from
// project_node and the tile sum from the same pairwise tree as the fused
// projection of the evolve kernels (tile slot k holds point base + k; thread t
// holds slots t, t + 256, t + 512, t + 768, so the tree's first two levels are
// in registers), so both give the same bits.  HBM-bound: 32 bytes of state read
// and 4 (FP32_MIXED) or 8 (FP64) bytes of map written per point.
constexpr int kProjThreads = 256;
constexpr int kProjPoints = kTilePoints / kProjThreads;
static_assert(kProjPoints == 4, "the first two tree levels are taken in registers");

template <int PREC>
__global__ void __launch_bounds__(kProjThreads, 3)
    project_kernel(const __grid_constant__ EvolveArgs args)
{
    __shared__ double red[kProjThreads];
    const int r = find_request(args);
    const ReqDesc &R = args.r[r];
    const int tile = static_cast<int>(blockIdx.x) - R.tile_begin;
    if (!tile_ok(R, tile, R.err))
        return;
    const int tid = threadIdx.x;
    const int64_t base = static_cast<int64_t>(tile) * kTilePoints;
    using Half = typename std::conditional<PREC == 1, float4, double2>::type;
    const Half *p0 = static_cast<const Half *>(R.state);
    const Half *p1 = p0 + R.n_points;
    Half u[kProjPoints], w[kProjPoints];
#pragma unroll
    for (int s = 0; s < kProjPoints; ++s) {
        const int64_t idx = base + s * kProjThreads + tid;
        if (idx < R.n_points) {
            u[s] = p0[idx];
            w[s] = p1[idx];
        }
    }
    // column and row of the first point, then stepped (no division per point)
    int64_t col = (base + tid) % R.nx, row = (base + tid) / R.nx;
    double v[kProjPoints];
#pragma unroll
    for (int s = 0; s < kProjPoints; ++s) {
        const int64_t idx = base + s * kProjThreads + tid;
        v[s] = 0.0;
        if (idx < R.n_points) {
            SpinorDF d;
            double ar, ai, br, bi;
            if constexpr (PREC == 1) {  // hi plane u, lo plane w
                d = SpinorDF{u[s].x, w[s].x, u[s].y, w[s].y, u[s].z, w[s].z, u[s].w, w[s].w};
                ar = static_cast<double>(u[s].x) + w[s].x;
                ai = static_cast<double>(u[s].y) + w[s].y;
                br = static_cast<double>(u[s].z) + w[s].z;
                bi = static_cast<double>(u[s].w) + w[s].w;
            } else {  // a plane u, b plane w
                ar = u[s].x; ai = u[s].y; br = w[s].x; bi = w[s].y;
                split_f64(ar, d.arh, d.arl);
                split_f64(ai, d.aih, d.ail);
                split_f64(br, d.brh, d.brl);
                split_f64(bi, d.bih, d.bil);
            }
            v[s] = project_node(R, col, row, d, ar, ai, br, bi);
            if (R.map) {
                if constexpr (PREC == 1)
                    static_cast<float *>(R.map)[idx] = static_cast<float>(v[s]);
                else
                    static_cast<double *>(R.map)[idx] = v[s];
            }
        }
        col += kProjThreads;
        while (col >= R.nx) {
            col -= R.nx;
            ++row;
        }
    }
    red[tid] = (v[0] + v[2]) + (v[1] + v[3]);  // tree levels 512 and 256
    __syncthreads();
    for (int s = kProjThreads / 2; s > 0; s >>= 1) {
        if (tid < s)
            red[tid] += red[tid + s];
        __syncthreads();
    }
    if (tid == 0)
        R.partials[tile] = red[0];
}

// One CTA per density: fixed-order per-thread sums, then a pairwise tree.
__global__ void __launch_bounds__(1024) finalize_kernel(const __grid_constant__ FinalizeArgs args)
{
    __shared__ double red[1024];
    const FinDesc &f = args.f[blockIdx.x];
    double acc = 0.0;
    for (int i = threadIdx.x; i < f.n_tiles; i += blockDim.x)
        acc += f.partials[i];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 512; s > 0; s >>= 1) {
        if (threadIdx.x < s)
            red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        *f.out = red[0] * f.scale;
}

// Time-parallel combination, one thread per momentum: psi <- M_s psi for s =
// 0 .. S-1 in time order, starting from v(p + A_in), all in FP64.
template <int PREC>
__global__ void __launch_bounds__(128) combine_kernel(const __grid_constant__ CombineArgs a)
{
    const int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (idx >= a.n_points)
        return;
    const double vs = a.valley > 0 ? 1.0 : -1.0;
    const double px = grid_node(a.px_min, a.hx, idx % a.nx);
    const double py = grid_node(a.py_min, a.hy, a.row0 + idx / a.nx);
    double ar, ai, br, bi;
    initial_spinor(px + a.a_in[0], py + a.a_in[1], vs, ar, ai, br, bi);
    const size_t slab = static_cast<size_t>(a.n_points) * 32;
    for (int s = 0; s < a.n_segments; ++s) {
        const unsigned char *seg = static_cast<const unsigned char *>(a.segs) + s * slab;
        double alr, ali, ber, bei;  // (alpha, beta): first column of M_s
        if constexpr (PREC == 1) {
            const float4 h = reinterpret_cast<const float4 *>(seg)[idx];
            const float4 l = reinterpret_cast<const float4 *>(seg)[a.n_points + idx];
            alr = static_cast<double>(h.x) + l.x;
            ali = static_cast<double>(h.y) + l.y;
            ber = static_cast<double>(h.z) + l.z;
            bei = static_cast<double>(h.w) + l.w;
        } else {
            const double2 c0 = reinterpret_cast<const double2 *>(seg)[idx];
            const double2 c1 = reinterpret_cast<const double2 *>(seg)[a.n_points + idx];
            alr = c0.x; ali = c0.y; ber = c1.x; bei = c1.y;
        }
        // a' = alpha a - conj(beta) b ; b' = beta a + conj(alpha) b
        const double nar = alr * ar - ali * ai - (ber * br + bei * bi);
        const double nai = alr * ai + ali * ar - (ber * bi - bei * br);
        const double nbr = ber * ar - bei * ai + (alr * br + ali * bi);
        const double nbi = ber * ai + bei * ar + (alr * bi - ali * br);
        ar = nar; ai = nai; br = nbr; bi = nbi;
    }
    if constexpr (PREC == 1) {
        float4 *hi = static_cast<float4 *>(a.state);
        float4 *lo = hi + a.n_points;
        const float h0 = static_cast<float>(ar), h1 = static_cast<float>(ai);
        const float h2 = static_cast<float>(br), h3 = static_cast<float>(bi);
        hi[idx] = make_float4(h0, h1, h2, h3);
        lo[idx] = make_float4(static_cast<float>(ar - h0), static_cast<float>(ai - h1),
                              static_cast<float>(br - h2), static_cast<float>(bi - h3));
    } else {
        double2 *pa = static_cast<double2 *>(a.state);
        pa[idx] = make_double2(ar, ai);
        pa[a.n_points + idx] = make_double2(br, bi);
    }
}

}  // namespace

cudaError_t launch_combine(const CombineArgs &args, int precision, cudaStream_t stream)
{
    if (args.n_points <= 0)
        return cudaSuccess;
    const int64_t blocks = (args.n_points + 127) / 128;
    if (precision == 1)
        combine_kernel<1><<<static_cast<unsigned>(blocks), 128, 0, stream>>>(args);
    else
        combine_kernel<0><<<static_cast<unsigned>(blocks), 128, 0, stream>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_evolve(const EvolveArgs &args, int precision, cudaStream_t stream)
{
    if (args.nreq <= 0 || args.total_tiles <= 0)
        return cudaSuccess;
    if (precision == 1)
        evolve_mixed_kernel<<<args.total_tiles, kMixedThreads, 0, stream>>>(args);
    else
        evolve_f64_kernel<<<args.total_tiles, kF64Threads, 0, stream>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_project(const EvolveArgs &args, int precision, cudaStream_t stream)
{
    if (args.nreq <= 0 || args.total_tiles <= 0)
        return cudaSuccess;
    if (precision == 1)
        project_kernel<1><<<args.total_tiles, kProjThreads, 0, stream>>>(args);
    else
        project_kernel<0><<<args.total_tiles, kProjThreads, 0, stream>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs &args, cudaStream_t stream)
{
    if (args.count <= 0)
        return cudaSuccess;
    finalize_kernel<<<args.count, 1024, 0, stream>>>(args);
    return cudaGetLastError();
}

}  // namespace dsp
