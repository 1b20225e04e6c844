// dsp_internal.h -- shared between the kernels and the host API (not installed).
//
// Launch descriptors are passed BY VALUE as __grid_constant__ kernel parameters,
// so queueing a launch needs no host-to-device copy and no allocation.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dsp {

// Points per CTA tile of the evolve kernels.
constexpr int kTilePoints = 1024;
// Row-strip tiles (ReqDesc::strips): columns per strip and rows per strip.
constexpr int kStripWidth = 256;
constexpr int kStripHeight = 4;
// Points per density partial sum (a granule: point index / kGranule); every CTA
// shape covers whole granules.
constexpr int kGranule = 256;
// Spinors per thread (independent momenta advanced together for ILP).
constexpr int kSpinorsPerThread = 2;
constexpr int kThreads = kTilePoints / kSpinorsPerThread;
// Requests one evolve launch can carry in its parameter block (96 x 232 bytes:
// within the 32 KB kernel-parameter limit).
constexpr int kMaxReqPerLaunch = 96;
// Device-side error bits (the launch's error word).
constexpr int kErrTimeout = 1;
constexpr int kErrBounds = 2;  // only set by builds with -DDSP_BOUNDS_CHECK
// Bound on one mbarrier wait, in nanoseconds of %globaltimer.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// Series levels: (degree of cos(theta) in x = theta^2, degree of
// sin(theta)/theta in x).  The host picks, per request, the lowest level whose
// truncation error, accumulated over all the request's steps at its largest
// phase step theta_max, stays below a fixed budget (see choose_level).
struct SeriesLevel {
    int dc, ds;
};
constexpr int kNumLevels = 8;
constexpr SeriesLevel kLevelsF32[kNumLevels] = {{2, 1}, {2, 2}, {3, 2}, {3, 3},
                                                 {4, 4}, {6, 6}, {9, 9}, {12, 12}};
constexpr SeriesLevel kLevelsF64[kNumLevels] = {{3, 3}, {4, 3}, {4, 4}, {5, 5},
                                                 {6, 6}, {8, 8}, {11, 11}, {16, 16}};

// FP32_MIXED step groups of EXACT and STRANG_XY divide each step by its real
// diagonal (the tan-normalised chain of the kernels) and need, in x = theta^2,
//   tan(theta)/theta = sum_k kTanSeries[k] x^k   (4^(k+1) (4^(k+1) - 1) |B_(2k+2)| / (2k+2)!)
//   sec(theta)       = sum_k kSecSeries[k] x^k   (|E_2k| / (2k)!)
// (B: Bernoulli numbers, E: Euler numbers), truncated after x^DT, DT one of
// kTanDegrees (the lowest whose truncation stays inside the series budget, see
// choose_tan_degree); and (1 + y)^(-1/2) = sum_k binom(-1/2, k) y^k truncated
// after y^kTanNormDegree(G) for the group's normalisation.
constexpr int kTanTerms = 8;
constexpr double kTanSeries[kTanTerms] = {1.0,
                                          1.0 / 3.0,
                                          2.0 / 15.0,
                                          17.0 / 315.0,
                                          62.0 / 2835.0,
                                          1382.0 / 155925.0,
                                          21844.0 / 6081075.0,
                                          929569.0 / 638512875.0};
constexpr double kSecSeries[kTanTerms] = {1.0,
                                          1.0 / 2.0,
                                          5.0 / 24.0,
                                          61.0 / 720.0,
                                          277.0 / 8064.0,
                                          50521.0 / 3628800.0,
                                          540553.0 / 95800320.0,
                                          199360981.0 / 87178291200.0};
constexpr int kNumTanDegrees = 5;
constexpr int kTanDegrees[kNumTanDegrees] = {1, 2, 3, 4, 6};

struct ReqDesc {
    // Per step, s = valley (valley K- steps as K+ on -P: its operator is K+'s at -P):
    //   EXACT, STRANG_XY: s*dt*A at the step midpoint, as float2 (FP32_MIXED) or
    //     double2 (FP64);
    //   MAGNUS4: s*dt*Abar, Abar = (A1 + A2)/2, and D = -(sqrt(3)/6) s*dt*(A2 - A1),
    //     A1, A2 at the two Gauss points: float4 (Abar_x, Abar_y, D_x, D_y) or two
    //     double2.
    const void *table;
    void *state;        // planes: FP32_MIXED float4 hi[n], float4 lo[n]; FP64 double2 a[n], double2 b[n]
    void *map;          // |c+|^2 output (float or double), or nullptr
    double *partials;   // one double per granule of kGranule points (written when projecting)
    int *err;           // the request's device error word (bits kErr*)
    const float2 *nodes_out;  // projection nodes p + A_out as FP32 hi/lo pairs: nx
                              // columns, then the grid's ny rows (see node_tables)
    double px_min, py_min, hx, hy;
    double dt;
    double a_in[2], a_out[2];
    int64_t n_points;
    int64_t step_begin, step_end;  // table entries [step_begin, step_end) this launch
    int32_t nx, ny;
    int32_t row0;     // global row index of the grid's first row (row bands; 0 otherwise)
    int32_t store_state;  // 1: write the spinor state back at the end of the launch
    int32_t scheme, valley, level;
    int32_t fresh;    // 1: start from v(p + A_in) instead of reading the state
    int32_t project;  // 1: project at the end (map + partials)
    int32_t tile_begin;  // first CTA of this request in the launch
    int32_t n_tiles;
    int32_t init_identity;  // with fresh: start from the column (1, 0) of the identity
                            // (the launch then computes the first column of the
                            // product of its steps' operators)
    int32_t group;   // FP32_MIXED (every scheme): the steps (G j, ..., G j + G - 1) of
                     // absolute index are multiplied into one operator before one
                     // compensated update; G = 1 (every step alone), 2, 4, 8 or kGroupMax
    int32_t tdeg;    // FP32_MIXED with G >= 2: degree DT of the tan (STRANG_XY: and
                     // sec) series, one of kTanDegrees
    int32_t withhold_first_copy;  // test hook: announce chunk 0 but never copy it, so the
                                  // bounded wait for it runs out (no fault, no hang)
    int32_t strips;  // 1: row strips (nx a multiple of kStripWidth): CTA tile b is rows
                     // strip_row0 + strip_h (b / (nx / 256)) .. + strip_h - 1, columns
                     // 256 (b % (nx / 256)) .. + 255; 0: CTA tile b is points
                     // 1024 b .. 1024 b + 1023
    int32_t strip_h;     // rows per strip: 4, or 2 for the strips that split a launch's
                         // last wave (the same points, half the work per CTA)
    int32_t strip_row0;  // first row of this descriptor's strips
    int32_t tail_split;  // 1: a launch of this request alone may split its last wave
                         // (host only; see split_last_wave)
    int64_t table_steps;          // entries in the table (checked by bounds-check builds)
};

// Steps are grouped (G = 16, 8, 4 or 2, the largest allowed) when G * theta_max
// stays within the scheme's group angle: the group's increment (U_G ... U_1 - I)
// psi then stays small next to psi, where the compensated (Fast2Sum) update
// keeps the state's rounding from accumulating.  The tan-normalised groups of
// EXACT and STRANG_XY take 0.27: on every point of the 2048^2 x 1e5-step LZS
// maps, raising their angle from 0.2 to 0.27 (groups of 16 instead of 8 on
// samples 1 and 2, of 8 instead of 4 on sample 6) left the largest FP32_MIXED
// error against FP64 where it was (2.13e-6 -> 2.18e-6, 1.76e-6 -> 1.96e-6,
// 4.32e-6 -> 4.27e-6), and a TwoSum update in place of Fast2Sum changed none of
// them.  MAGNUS4 groups (tan-normalised too, with the sigma_z part in the chain)
// keep 0.2, the angle at which they were measured.
constexpr int kGroupMax = 16;
constexpr double kGroupAngleTan = 0.27;
constexpr double kGroupAngleMagnus = 0.2;

// Degree of the (1 + y)^(-1/2) series that normalises a tan-normalised group of
// G steps: y = det W - 1 = prod(1 + tan^2 theta_k) - 1 ~ G theta_max^2 <=
// kGroupAngleTan^2 / G (with 5% to spare for the tan^2 and the product); the
// lowest degree whose first omitted term |binom(-1/2, d + 1)| y^(d + 1) stays
// below 1e-14 (G = 16, 8, 4, 2: degree 5, 6, 7, 9).
__host__ __device__ constexpr int kTanNormDegree(int G)
{
    const double y = 1.05 * kGroupAngleTan * kGroupAngleTan / G;
    double c = 1.0, yk = 1.0;  // |binom(-1/2, k)|, y^k
    for (int k = 1; k < 16; ++k) {
        c *= static_cast<double>(2 * k - 1) / static_cast<double>(2 * k);
        yk *= y;
        if (c * yk <= 1e-14)
            return k - 1;
    }
    return 15;
}
static_assert(kTanNormDegree(16) == 5 && kTanNormDegree(8) == 6 && kTanNormDegree(4) == 7 &&
                  kTanNormDegree(2) == 9,
              "normalisation degrees of the tan-normalised groups");

static_assert(sizeof(ReqDesc) * kMaxReqPerLaunch + 64 < 32764, "kernel parameter limit");

struct EvolveArgs {
    int32_t nreq;
    int32_t total_tiles;
    ReqDesc r[kMaxReqPerLaunch];
};

struct FinDesc {
    const double *partials;
    int64_t n_parts;  // granule partial sums
    double scale;     // 4/(2 pi)^2 * hx * hy
    double *out;      // device double
};

constexpr int kMaxFinPerLaunch = 64;
struct FinalizeArgs {
    int32_t count;
    int32_t pad;
    FinDesc f[kMaxFinPerLaunch];
};

// Combines time segments: psi = M_{S-1} ... M_0 v(p + A_in) per point, where M_s
// is the SU(2) matrix [[alpha, -conj(beta)], [beta, conj(alpha)]] whose first
// column (alpha, beta) segment s left in its slab of `segs`; writes psi into
// `state` in the grid's layout.  FP64 arithmetic for both precisions.
struct CombineArgs {
    const void *segs;  // S slabs of 32 * n_points bytes, in the state layout
    void *state;
    int64_t n_points;
    int32_t n_segments;
    int32_t nx;
    double px_min, py_min, hx, hy;
    double a_in[2];
    int32_t valley;
    int32_t row0;  // global row index of the grid's first row
};

// Evolve launches, one kernel per kind of request: FP64 or FP32_MIXED, on
// contiguous tiles (strips == 0) or on row strips (strips == 1).  Every request
// in args must be of that kind.
cudaError_t launch_evolve_f64(const EvolveArgs &args, cudaStream_t stream);
cudaError_t launch_evolve_f64_strip(const EvolveArgs &args, cudaStream_t stream);
cudaError_t launch_evolve_mixed(const EvolveArgs &args, cudaStream_t stream);
// FP32_MIXED row strips: one kernel per scheme and strip height (every request in
// args has that scheme and strip_h).
cudaError_t launch_evolve_strip(const EvolveArgs &args, int scheme, int strip_h,
                                cudaStream_t stream);
// CTAs of the 4-row strip kernel of a precision (and FP32_MIXED scheme) that one
// SM holds at once.
cudaError_t strip_ctas_per_sm(int precision, int scheme, int *ctas);
// Projection only, of states already on the device: every request in args has
// step_begin == step_end, project == 1, fresh == 0 and a node table.
cudaError_t launch_project(const EvolveArgs &args, int precision, cudaStream_t stream);
cudaError_t launch_finalize(const FinalizeArgs &args, cudaStream_t stream);
cudaError_t launch_combine(const CombineArgs &args, int precision, cudaStream_t stream);

}  // namespace dsp
