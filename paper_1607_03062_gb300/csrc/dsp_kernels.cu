// dsp_kernels.cu -- the FP64 evolve kernel, the projection-only kernel, the
// density finalisation and the time-segment combination.  Shared device code
// (and the description of the method and of the GB300 design) is in
// dsp_device.cuh.

#include "dsp_device.cuh"

namespace dsp {
namespace {

// ---------------------------------------------------------------------------
// FP64 step
// ---------------------------------------------------------------------------

struct F64Point {
    double ar, ai, br, bi;
    double tx, ty;  // dt * p (times the valley sign)
};

// ---------------------------------------------------------------------------
// The FP64 EXACT step with its small parts in double-float.
//
// GB300's FP64 pipe runs at 1/64 of the FP32 rate (a warp's DFMA holds a
// scheduler's FP64 unit for ~64 cycles), so only what must accumulate in FP64 is
// done there: the update psi <- psi + m psi - (q conj ...) and q = dt P + s1 dt P.
// The small parts m = cos(theta) - 1 and s1 = sin(theta)/theta - 1 of theta^2 =
// |dt P|^2 are evaluated in double-float FP32 arithmetic (pairs of floats, ~2^-46
// relative): being small (~theta^2/2, ~theta^2/6), they come out to ~1e-19
// absolute, far below an FP64 ulp of the state, so the step is FP64-accurate.
// FP64 operations per spinor-step: 2 (dt P) + 2 (m, s1 to double) + 2 (q) + 12
// (update) = 18 instead of 18 + dc + ds; the ~100 FP32 operations of the series
// issue beside them.
// ---------------------------------------------------------------------------

// dt P squared as a float pair, from the double (split exactly into hi + lo).
__device__ __forceinline__ float2 square_df(double P)
{
    float h, l;
    split_f64(P, h, l);
    const float p = __fmul_rn(h, h);
    const float e = __fmaf_rn(__fadd_rn(h, h), l, __fmaf_rn(h, h, -p));
    const float sh = __fadd_rn(p, e);
    return make_float2(sh, __fadd_rn(e, -__fadd_rn(sh, -p)));
}

// sum_{k=K..D} c_k x^(k-K) in double-float, c_k = (-1)^k / (2k + ODD)!.
template <int D, int K, int ODD>
__device__ __forceinline__ void horner_df(float xh, float xl, float &th, float &tl)
{
    constexpr DFConst c = df_const(((K & 1) ? -1.0 : 1.0) * inv_factorial<2 * K + ODD>());
    if constexpr (K == D) {
        th = c.h;
        tl = c.l;
    } else {
        float uh, ul;
        horner_df<D, K + 1, ODD>(xh, xl, uh, ul);
        df_mul(xh, xl, uh, ul, th, tl);
        df_add(th, tl, c.h, c.l);
    }
}

// The FP64 EXACT step: dt P = (Px, Py), their squares as float pairs.
template <int DC, int DS>
__device__ __forceinline__ void step_f64_exact(F64Point &s, double Px, double Py, float2 px2,
                                               float2 py2)
{
    float xh = px2.x, xl = px2.y;
    df_add(xh, xl, py2.x, py2.y);  // theta^2
    float th, tl, mh, ml, sh, sl;
    horner_df<DC, 1, 0>(xh, xl, th, tl);  // (cos(theta) - 1) / theta^2
    df_mul(xh, xl, th, tl, mh, ml);
    horner_df<DS, 1, 1>(xh, xl, th, tl);  // (sin(theta)/theta - 1) / theta^2
    df_mul(xh, xl, th, tl, sh, sl);
    const double m = df_to_f64(mh, ml), s1 = df_to_f64(sh, sl);
    const double qr = fma(s1, Py, Py), qi = fma(s1, Px, Px);
    // a' = a + m a - q b ; b' = b + m b + conj(q) a, q = qr + i qi
    const double nar = fma(m, s.ar, fma(-qr, s.br, fma(qi, s.bi, s.ar)));
    const double nai = fma(m, s.ai, fma(-qr, s.bi, fma(-qi, s.br, s.ai)));
    const double nbr = fma(m, s.br, fma(qr, s.ar, fma(qi, s.ai, s.br)));
    const double nbi = fma(m, s.bi, fma(qr, s.ai, fma(-qi, s.ar, s.bi)));
    s.ar = nar; s.ai = nai; s.br = nbr; s.bi = nbi;
}

// psi <- U psi for U = [[c, -q], [conj(q), c]] (STRANG_XY), in FP64.
__device__ __forceinline__ void apply_f64(F64Point &s, double c, double qr, double qi)
{
    const double nar = fma(c, s.ar, fma(-qr, s.br, qi * s.bi));
    const double nai = fma(c, s.ai, fma(-qr, s.bi, -(qi * s.br)));
    const double nbr = fma(c, s.br, fma(qr, s.ar, qi * s.ai));
    const double nbi = fma(c, s.bi, fma(qr, s.ai, -(qi * s.ar)));
    s.ar = nar; s.ai = nai; s.br = nbr; s.bi = nbi;
}

template <int SCHEME, int DC, int DS>
__device__ __forceinline__ void step_f64(F64Point &s, double2 a, double2 d)
{
    const double Px = s.tx + a.x, Py = s.ty + a.y;  // dt * P (times the valley sign)
    if constexpr (SCHEME == 0) {
        step_f64_exact<DC, DS>(s, Px, Py, square_df(Px), square_df(Py));
        return;
    }
    double c, qr, qi, qz = 0.0;
    if constexpr (SCHEME == 1) {
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
    if constexpr (SCHEME == 2) {
        const double nar = fma(c, s.ar, fma(qz, s.ai, fma(-qr, s.br, qi * s.bi)));
        const double nai = fma(c, s.ai, fma(-qz, s.ar, fma(-qr, s.bi, -(qi * s.br))));
        const double nbr = fma(c, s.br, fma(-qz, s.bi, fma(qr, s.ar, qi * s.ai)));
        const double nbi = fma(c, s.bi, fma(qz, s.br, fma(qr, s.ai, -(qi * s.ar))));
        s.ar = nar; s.ai = nai; s.br = nbr; s.bi = nbi;
    } else {
        apply_f64(s, c, qr, qi);
    }
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

    float2 *red = reinterpret_cast<float2 *>(smem);
#pragma unroll
    for (int s = 0; s < S; ++s) {
        const int64_t idx = base + s * kThreads + tid;
        float2 c = make_float2(0.0f, 0.0f);
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
                c = store_point<0>(R.map, idx, project_node<0>(R, idx % R.nx, idx / R.nx, v));
            }
        }
        if (R.project)
            red[s * kThreads + tid] = c;
    }
    if (R.project)
        granule_sums(red, kTilePoints / kGranule, R.partials, (R.n_points + kGranule - 1) / kGranule,
                     [&](int g) { return base / kGranule + g; });
}

// ---------------------------------------------------------------------------
// FP64 EXACT and STRANG_XY on row strips (grids whose nx is a multiple of 256)
//
// The tiling of the FP32_MIXED strips (a CTA owns 4 rows x 256 columns, thread
// t column c0 + t of each row): dt P_x is formed once per thread and step for
// its 4 spinors, and the dt P_y parts of a step once per row into a table in
// shared memory (EXACT: dt P_y and dt P_y^2 as a float pair; STRANG_XY:
// cos(dt P_y) and dt P_y sinc(dt P_y)).  Every operation on a point is
// step_f64's, so each point's result is bitwise the same on either tiling; FP64
// work per spinor-step drops from 18 to 16.25 (EXACT).
// ---------------------------------------------------------------------------

constexpr int kStrip64Threads = kStripWidth;
constexpr int kStrip64Rows = kStripHeight;
constexpr int kStrip64Stage = 4096;                 // bytes per staged table chunk
constexpr int kStrip64Chunk = kStrip64Stage / 16;  // steps per chunk (double2 entries)
static_assert(kStrip64Threads * kStrip64Rows == kTilePoints, "a strip tile holds kTilePoints points");
static_assert(kStrip64Threads == kGranule, "a strip row is one density granule");

struct Strip64Smem {
    unsigned char stage[2][kStrip64Stage];     // bulk-copied table entries (dt A_x, dt A_y)
    double2 rows[kStrip64Chunk][kStrip64Rows];  // per step and row: see strip64_row
    double ax[kStrip64Chunk];                   // per step: dt A_x
};
static_assert(sizeof(Strip64Smem) <= 48 * 1024, "static shared memory of one CTA");
static_assert(sizeof(Strip64Smem) >= kTilePoints * sizeof(float2), "holds the density slots");

// The row part of a step from dt P_y, as step_f64 forms it:
//   EXACT {P_y, (P_y^2 as a float pair, in the second double's bits)};
//   STRANG_XY {cos(P_y), P_y * sinc(P_y)} (b = dt P_y).
template <int SCHEME, int DC, int DS>
__device__ __forceinline__ double2 strip64_row(double Py)
{
    if constexpr (SCHEME == 0) {
        const float2 p2 = square_df(Py);
        const unsigned long long bits =
            (static_cast<unsigned long long>(__float_as_uint(p2.y)) << 32) | __float_as_uint(p2.x);
        return make_double2(Py, __longlong_as_double(static_cast<long long>(bits)));
    } else {
        const double xy = Py * Py;
        return make_double2(cos_f64<DC>(xy), Py * sinc_f64<DS>(xy));
    }
}

// One step of the thread's H spinors (step_f64's operations; SCHEME 0 EXACT, 1
// STRANG_XY).
template <int SCHEME, int DC, int DS, int H>
__device__ __forceinline__ void strip64_step(F64Point (&pt)[H], double tx, double ax,
                                             const double2 *rows)
{
    const double Px = tx + ax;  // dt * P_x (times the valley sign)
    if constexpr (SCHEME == 0) {
        const float2 px2 = square_df(Px);
#pragma unroll
        for (int k = 0; k < H; ++k) {
            const double2 r = rows[k];
            const unsigned long long bits = static_cast<unsigned long long>(__double_as_longlong(r.y));
            const float2 py2 = make_float2(__uint_as_float(static_cast<unsigned int>(bits)),
                                           __uint_as_float(static_cast<unsigned int>(bits >> 32)));
            step_f64_exact<DC, DS>(pt[k], Px, r.x, px2, py2);
        }
        return;
    }
    // STRANG_XY: the column's cos(dt P_x) and dt P_x sinc(dt P_x), then per row
    const double xx = Px * Px;
    const double cxx = cos_f64<DC>(xx);
    const double sxx = Px * sinc_f64<DS>(xx);
#pragma unroll
    for (int k = 0; k < H; ++k) {
        const double2 r = rows[k];
        apply_f64(pt[k], r.x * cxx, r.y, r.x * sxx);
    }
}

// A strip tile of H rows (4 normally, 2 for the strips that split a launch's last
// wave, see ReqDesc::strip_h).
template <int SCHEME, int DC, int DS, int H>
__device__ void body_strip_f64(const ReqDesc &R, int tile, unsigned char *smem, uint64_t *bars,
                               int *err)
{
    Strip64Smem &sm = *reinterpret_cast<Strip64Smem *>(smem);
    const int tid = threadIdx.x;
    const int ncb = R.nx / kStrip64Threads;
    const int rb = tile / ncb, cb = tile - rb * ncb;
    const int64_t row_first = R.strip_row0 + static_cast<int64_t>(rb) * H;
    const int64_t col = static_cast<int64_t>(cb) * kStrip64Threads + tid;
    const double vs = R.valley > 0 ? 1.0 : -1.0;
    double2 *a_plane = static_cast<double2 *>(R.state);
    double2 *b_plane = a_plane + R.n_points;
    const double px = grid_node(R.px_min, R.hx, col);
    const double tx = vs * (R.dt * px);  // valley K- is stepped as K+ on -P
    F64Point pt[H];
#pragma unroll
    for (int k = 0; k < H; ++k) {
        const int64_t row = row_first + k;
        const bool valid = row < R.ny;  // the last strip of a grid may hang over its end
        const int64_t idx = row * R.nx + col;
        const double py = grid_node(R.py_min, R.hy, R.row0 + row);
        pt[k].tx = tx;
        pt[k].ty = vs * (R.dt * py);
        if (R.fresh || !valid) {
            if (R.init_identity) {
                pt[k].ar = 1.0; pt[k].ai = 0.0; pt[k].br = 0.0; pt[k].bi = 0.0;
            } else {
                initial_spinor(px + R.a_in[0], py + R.a_in[1], vs, pt[k].ar, pt[k].ai, pt[k].br,
                               pt[k].bi);
            }
        } else {
            const double2 a = a_plane[idx], b = b_plane[idx];
            pt[k].ar = a.x; pt[k].ai = a.y; pt[k].br = b.x; pt[k].bi = b.y;
        }
    }

    using St = Stager<double2, kStrip64Stage>;
    const int64_t b_al = R.step_begin;  // 16-byte entries: every step starts on a boundary
    bool ok = table_range_ok(R, b_al, err);
    if (ok) {
        St st{&sm.stage[0][0], bars, static_cast<const double2 *>(R.table) + b_al,
              R.step_end - b_al, 0};
        st.withhold_first = R.withhold_first_copy;
        if (R.step_end <= R.step_begin)
            st.nsteps = 0;
        st.nchunks = static_cast<int>((st.nsteps + St::kCh - 1) / St::kCh);
        if (tid == 0) {
            if (st.nchunks > 0) st.issue(0);
            if (st.nchunks > 1) st.issue(1);
        }
        for (int c = 0; c < st.nchunks; ++c) {
            const bool arrived = mbar_wait_bounded(&bars[c & 1], (c >> 1) & 1);
            if (!__syncthreads_and(arrived)) {
                if (tid == 0)
                    st.on_timeout(c, err);
                ok = false;
                break;
            }
            const double2 *tb = st.stage(c);
            const int len = st.chunk_len(c);
            // the row table of this chunk, from dt P_y = s dt p_y + s dt A_y
            for (int j = tid; j < len; j += blockDim.x) {
                const double2 a = tb[j];
                sm.ax[j] = a.x;
#pragma unroll
                for (int k = 0; k < H; ++k)
                    sm.rows[j][k] = strip64_row<SCHEME, DC, DS>(pt[k].ty + a.y);
            }
            __syncthreads();  // the table is built and stage c & 1 is free again
            if (tid == 0 && c + 2 < st.nchunks)
                st.issue(c + 2);
#pragma unroll 2
            for (int j = 0; j < len; ++j)
                strip64_step<SCHEME, DC, DS, H>(pt, tx, sm.ax[j], sm.rows[j]);
            __syncthreads();  // everyone is done with the row table
        }
    }
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
                a_plane[idx] = make_double2(pt[k].ar, pt[k].ai);
                b_plane[idx] = make_double2(pt[k].br, pt[k].bi);
            }
            if (R.project) {
                SpinorDF v;
                split_f64(pt[k].ar, v.arh, v.arl);
                split_f64(pt[k].ai, v.aih, v.ail);
                split_f64(pt[k].br, v.brh, v.brl);
                split_f64(pt[k].bi, v.bih, v.bil);
                c = store_point<0>(R.map, idx, project_node<0>(R, col, row, v));
            }
        }
        if (R.project)
            red[k * kGranule + tid] = c;
    }
    if (R.project)  // granule of strip row k: row (row_first + k), columns from cb * 256
        granule_sums(red, H, R.partials, (R.n_points + kGranule - 1) / kGranule,
                     [&](int g) { return (row_first + g) * ncb + cb; });
}

template <int SCHEME, int L>
__device__ __forceinline__ void dispatch_strip_f64(const ReqDesc &R, int tile, unsigned char *smem,
                                                   uint64_t *bars, int *err)
{
    if (R.level == L || L + 1 == kNumLevels) {
        constexpr int DC = kLevelsF64[L].dc, DS = kLevelsF64[L].ds;
        if (R.strip_h == 2)
            body_strip_f64<SCHEME, DC, DS, 2>(R, tile, smem, bars, err);
        else
            body_strip_f64<SCHEME, DC, DS, kStrip64Rows>(R, tile, smem, bars, err);
    } else if constexpr (L + 1 < kNumLevels) {
        dispatch_strip_f64<SCHEME, L + 1>(R, tile, smem, bars, err);
    }
}

// Block-uniform dispatch on the request's series level (compile-time degrees).
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

__global__ void __launch_bounds__(kStrip64Threads, 2)
    evolve_f64_strip_kernel(const __grid_constant__ EvolveArgs args)
{
    __shared__ __align__(128) unsigned char smem[sizeof(Strip64Smem)];
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
        dispatch_strip_f64<0, 0>(R, tile, smem, bars, R.err);
    else
        dispatch_strip_f64<1, 0>(R, tile, smem, bars, R.err);
}

// Projection of a state already on the device (a launch with no steps).  HBM
// streaming with no CTA-wide barrier: every warp works on its own granules
// (256 points: the density's partial-sum unit) through its own ring of
// shared-memory buffers (ProjShape).  Lane 0 queues both state planes of a
// granule (2 x 4 KB) by 1-D bulk copy (cp.async.bulk) completing on the
// buffer's mbarrier; the copies of the other warps on the SM are in flight
// while one projects (with two buffers a warp also overlaps its own).
// Lane l holds the granule's points l, l + 32, ..., l + 224: the pairwise tree
// of granule_sums (slot j plus slot j + s for s = 128, ..., 1) then takes its
// first three levels inside each lane and the last five across lanes by
// shuffles, the same pairs in the same order, and each point's value comes
// from project_node and store_point as in the evolve kernels, so both give the
// same bits.  Per point: 32 bytes of state read, 4 (FP32_MIXED) or 8 (FP64)
// bytes of map written; FP64-pipe work is one add per point for an FP64 map,
// none for FP32_MIXED.
// Shape per precision: warps per CTA (one CTA per SM) and buffers per warp's
// ring.  Measured on a 4096^2 state (us per launch, FP32_MIXED / FP64): 12
// warps x 2 buffers 109.5 / 258.7, 16 x 1 - / 242.1, 24 x 1 105.7 / 214.0: many
// warps with one buffer each hide both the copies and the latency of the
// double-float arithmetic best.
#ifndef DSP_PROJ32_WARPS
#define DSP_PROJ32_WARPS 24
#endif
#ifndef DSP_PROJ32_BUFS
#define DSP_PROJ32_BUFS 1
#endif
#ifndef DSP_PROJ64_WARPS
#define DSP_PROJ64_WARPS 24
#endif
#ifndef DSP_PROJ64_BUFS
#define DSP_PROJ64_BUFS 1
#endif
template <int PREC>
struct ProjShape {
    static constexpr int warps = PREC == 1 ? DSP_PROJ32_WARPS : DSP_PROJ64_WARPS;
    static constexpr int bufs = PREC == 1 ? DSP_PROJ32_BUFS : DSP_PROJ64_BUFS;
    static constexpr int threads = 32 * warps;
    static constexpr int plane = kGranule * 16;          // bytes of one state plane of a granule
    static constexpr int warp_bytes = bufs * 2 * plane;  // a warp's ring
    static constexpr int smem = warps * (warp_bytes + bufs * 8);
};
constexpr int kProjPer = kGranule / 32;  // points per lane and granule
static_assert(kTilePoints % kGranule == 0, "tiles hold whole granules");

template <int PREC>
__global__ void __launch_bounds__(ProjShape<PREC>::threads, 1)
    project_kernel(const __grid_constant__ EvolveArgs args)
{
    using Sh = ProjShape<PREC>;
    constexpr int kProjPlane = Sh::plane;
    constexpr int NB = Sh::bufs;
    extern __shared__ __align__(128) unsigned char proj_dyn[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned char *buf = proj_dyn + w * Sh::warp_bytes;  // [buffer][plane][kProjPlane]
    uint64_t *bars = reinterpret_cast<uint64_t *>(proj_dyn + Sh::warps * Sh::warp_bytes) + NB * w;
    constexpr int kGranPerTile = kTilePoints / kGranule;
    const int total = args.total_tiles * kGranPerTile;  // granules of the launch
    const int wid = blockIdx.x * Sh::warps + w, nw = gridDim.x * Sh::warps;
    if (lane == 0) {
        for (int b = 0; b < NB; ++b)
            mbar_init(&bars[b], 1);
        fence_mbar_init();
    }
    __syncwarp();
    // lane 0 queues both planes of granule Gi into buffer b (whole 16-byte points);
    // a granule past the end of its grid completes its phase empty
    const auto issue = [&](int Gi, int b) {
        const int T = Gi / kGranPerTile;
        const ReqDesc &R = args.r[find_request(args, T)];
        const int64_t base = static_cast<int64_t>(T - R.tile_begin) * kTilePoints +
                             static_cast<int64_t>(Gi % kGranPerTile) * kGranule;
        const int64_t left = R.n_points - base;
        const uint32_t bytes =
            left <= 0 ? 0u : 16u * static_cast<uint32_t>(left < kGranule ? left : kGranule);
        mbar_arrive_expect_tx(&bars[b], 2 * bytes);
        if (bytes > 0) {
            const unsigned char *st = static_cast<const unsigned char *>(R.state);
            unsigned char *dst = buf + b * 2 * kProjPlane;
            bulk_load(dst, st + 16 * base, bytes, &bars[b]);
            bulk_load(dst + kProjPlane, st + 16 * (R.n_points + base), bytes, &bars[b]);
        }
    };
    if (lane == 0)
        for (int b = 0; b < NB; ++b)
            if (wid + b * nw < total)
                issue(wid + b * nw, b);
    int k = 0;
    for (int Gi = wid; Gi < total; Gi += nw, ++k) {
        const int b = k % NB;
        const int T = Gi / kGranPerTile;
        const ReqDesc &R = args.r[find_request(args, T)];
        const bool arrived = mbar_wait_bounded(&bars[b], (k / NB) & 1);
        if (!__all_sync(0xffffffffu, arrived)) {
            if (lane == 0) {  // flag it; give the copies still queued a bounded chance to
                              // land before the warp leaves
                atomicOr(R.err, kErrTimeout);
                for (int j = 1; j < NB; ++j)
                    if (Gi + j * nw < total)
                        (void)mbar_wait_bounded(&bars[(k + j) % NB], ((k + j) / NB) & 1);
            }
            return;
        }
        const int tile = T - R.tile_begin;
        if (tile_ok(R, tile, R.err)) {
            const int64_t gbase = static_cast<int64_t>(tile) * kTilePoints +
                                  static_cast<int64_t>(Gi % kGranPerTile) * kGranule;
            // column and row of the granule's first point (one division per granule)
            int64_t col0 = 0, row0 = 0;
            if (lane == 0) {
                col0 = gbase % R.nx;
                row0 = gbase / R.nx;
            }
            col0 = __shfl_sync(0xffffffffu, col0, 0);
            row0 = __shfl_sync(0xffffffffu, row0, 0);
            const unsigned char *src = buf + b * 2 * kProjPlane;
            // the state of the lane's point l = lane + 32 i, as hi/lo pairs
            const auto spinor = [&](int l) {
                SpinorDF d;
                if constexpr (PREC == 1) {  // hi plane, lo plane
                    const float4 u = reinterpret_cast<const float4 *>(src)[l];
                    const float4 q = reinterpret_cast<const float4 *>(src + kProjPlane)[l];
                    d = SpinorDF{u.x, q.x, u.y, q.y, u.z, q.z, u.w, q.w};
                } else {  // a plane, b plane
                    const double2 u = reinterpret_cast<const double2 *>(src)[l];
                    const double2 q = reinterpret_cast<const double2 *>(src + kProjPlane)[l];
                    split_f64(u.x, d.arh, d.arl);
                    split_f64(u.y, d.aih, d.ail);
                    split_f64(q.x, d.brh, d.brl);
                    split_f64(q.y, d.bih, d.bil);
                }
                return d;
            };
            float2 v[kProjPer];
            if (gbase + kGranule <= R.n_points && col0 + kGranule <= R.nx) {
                // a whole granule inside one row (every grid whose nx is a multiple of 256):
                // one row node, the column nodes loaded up front, no bounds to check
                const float2 cy = R.nodes_out[R.nx + row0];
                float2 cx[kProjPer];
#pragma unroll
                for (int i = 0; i < kProjPer; ++i)
                    cx[i] = R.nodes_out[col0 + lane + 32 * i];
#pragma unroll
                for (int i = 0; i < kProjPer; ++i) {
                    const int l = lane + 32 * i;
                    v[i] = store_point<PREC>(
                        R.map, gbase + l,
                        project_node_at<PREC>(R, cx[i], cy, col0 + l, row0, spinor(l)));
                }
            } else {
                int64_t col = col0 + lane, row = row0;
                while (col >= R.nx) {
                    col -= R.nx;
                    ++row;
                }
#pragma unroll
                for (int i = 0; i < kProjPer; ++i) {
                    const int l = lane + 32 * i;
                    const int64_t idx = gbase + l;
                    v[i] = make_float2(0.0f, 0.0f);
                    if (idx < R.n_points)
                        v[i] = store_point<PREC>(R.map, idx,
                                                 project_node<PREC>(R, col, row, spinor(l)));
                    col += 32;
                    while (col >= R.nx) {
                        col -= R.nx;
                        ++row;
                    }
                }
            }
            // granule_sums' tree: s = 128, 64, 32 within the lane, s = 16 .. 1 across lanes
#pragma unroll
            for (int s = kProjPer / 2; s > 0; s >>= 1)
#pragma unroll
                for (int i = 0; i < s; ++i)
                    df_add(v[i].x, v[i].y, v[i + s].x, v[i + s].y);
#pragma unroll
            for (int s = 16; s > 0; s >>= 1) {
                const float h = __shfl_down_sync(0xffffffffu, v[0].x, s);
                const float l = __shfl_down_sync(0xffffffffu, v[0].y, s);
                if (lane < s)
                    df_add(v[0].x, v[0].y, h, l);
            }
            const int64_t gi = gbase / kGranule;
            if (lane == 0 && gi < (R.n_points + kGranule - 1) / kGranule)
                R.partials[gi] = df_to_f64(v[0].x, v[0].y);
        }
        __syncwarp();  // the warp is done with buffer b
        if (lane == 0 && Gi + NB * nw < total)
            issue(Gi + NB * nw, b);
    }
}

// One CTA per density: fixed-order per-thread sums of the granule partials,
// then a pairwise tree.
__global__ void __launch_bounds__(1024) finalize_kernel(const __grid_constant__ FinalizeArgs args)
{
    __shared__ double red[1024];
    const FinDesc &f = args.f[blockIdx.x];
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < f.n_parts; i += blockDim.x)
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

cudaError_t launch_evolve_f64(const EvolveArgs &args, cudaStream_t stream)
{
    if (args.nreq <= 0 || args.total_tiles <= 0)
        return cudaSuccess;
    evolve_f64_kernel<<<args.total_tiles, kF64Threads, 0, stream>>>(args);
    return cudaGetLastError();
}

// The FP32_MIXED strip kernels, one object of dsp_strip.cu each.
cudaError_t strip_ctas_per_sm_s0_np2(int *ctas);
cudaError_t strip_ctas_per_sm_s1_np2(int *ctas);
cudaError_t strip_ctas_per_sm_s2_np2(int *ctas);
cudaError_t launch_evolve_strip_s0_np2(const EvolveArgs &args, cudaStream_t stream);
cudaError_t launch_evolve_strip_s0_np1(const EvolveArgs &args, cudaStream_t stream);
cudaError_t launch_evolve_strip_s1_np2(const EvolveArgs &args, cudaStream_t stream);
cudaError_t launch_evolve_strip_s1_np1(const EvolveArgs &args, cudaStream_t stream);
cudaError_t launch_evolve_strip_s2_np2(const EvolveArgs &args, cudaStream_t stream);
cudaError_t launch_evolve_strip_s2_np1(const EvolveArgs &args, cudaStream_t stream);

cudaError_t strip_ctas_per_sm(int precision, int scheme, int *ctas)
{
    if (precision == 1)
        return scheme == 0   ? strip_ctas_per_sm_s0_np2(ctas)
               : scheme == 1 ? strip_ctas_per_sm_s1_np2(ctas)
                             : strip_ctas_per_sm_s2_np2(ctas);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, evolve_f64_strip_kernel,
                                                         kStrip64Threads, 0);
}

cudaError_t launch_evolve_strip(const EvolveArgs &args, int scheme, int strip_h,
                                cudaStream_t stream)
{
    const bool half = strip_h == 2;
    if (scheme == 0)
        return half ? launch_evolve_strip_s0_np1(args, stream)
                    : launch_evolve_strip_s0_np2(args, stream);
    if (scheme == 1)
        return half ? launch_evolve_strip_s1_np1(args, stream)
                    : launch_evolve_strip_s1_np2(args, stream);
    return half ? launch_evolve_strip_s2_np1(args, stream) : launch_evolve_strip_s2_np2(args, stream);
}

cudaError_t launch_evolve_f64_strip(const EvolveArgs &args, cudaStream_t stream)
{
    if (args.nreq <= 0 || args.total_tiles <= 0)
        return cudaSuccess;
    evolve_f64_strip_kernel<<<args.total_tiles, kStrip64Threads, 0, stream>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_project(const EvolveArgs &args, int precision, cudaStream_t stream)
{
    if (args.nreq <= 0 || args.total_tiles <= 0)
        return cudaSuccess;
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    // the warps' rings are above the 48 KB a kernel gets without asking
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(project_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 ProjShape<1>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(project_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 ProjShape<0>::smem);
    if (e != cudaSuccess)
        return e;
    // one CTA per SM, no more warps than granules
    const int granules = args.total_tiles * (kTilePoints / kGranule);
    const int warps = precision == 1 ? ProjShape<1>::warps : ProjShape<0>::warps;
    const int need = (granules + warps - 1) / warps;
    const int grid = need < sms ? need : sms;
    if (precision == 1)
        project_kernel<1><<<grid, ProjShape<1>::threads, ProjShape<1>::smem, stream>>>(args);
    else
        project_kernel<0><<<grid, ProjShape<0>::threads, ProjShape<0>::smem, stream>>>(args);
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
