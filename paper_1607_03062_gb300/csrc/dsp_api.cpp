// dsp_api.cpp -- host side of the C ABI declared in include/dsp.h: grid
// handles, pulse tables, launches, the density reduction, the pulse sampler and
// the continuous-batching server.
//
// The hot path runs entirely in the kernels of dsp_kernels.cu; this file only
// validates, lays out the per-step table in the layout the kernels read, and
// queues work on the caller's CUDA stream.

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include "dsp.h"
#include "dsp_internal.h"

using dsp::EvolveArgs;
using dsp::FinalizeArgs;
using dsp::ReqDesc;

namespace {

constexpr double kPi = 3.14159265358979323846;

// Named host-side range for timeline profilers (NVTX; free when none is attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

struct DeviceScalars {
    double density;
    int err;
    int pad;
};

}  // namespace

struct dsp_grid {
    int32_t nx = 0, ny = 0, precision = 0, scheme = 0, valley = 1;
    int32_t row0 = 0, ny_total = 0;  // rows [row0, row0 + ny) of an ny_total-row grid
    double px_min = 0, px_max = 0, py_min = 0, py_max = 0, hx = 0, hy = 0;
    int64_t n_points = 0;
    int32_t n_tiles = 0;  // CTAs of an evolve launch
    int64_t n_parts = 0;  // density partial sums (granules of dsp::kGranule points)
    cudaStream_t stream = nullptr;

    void *state = nullptr;
    bool owns_state = false;
    void *table = nullptr;
    int64_t table_cap = 0;  // entries
    double *partials = nullptr;
    DeviceScalars *scal = nullptr;
    float2 *nodes = nullptr;  // projection nodes s (p + A_out), FP32 hi/lo: nx columns, ny rows
    void *own_map = nullptr;  // used by dsp_solve when the caller passes no map
    void *seg_buf = nullptr;  // time-segment columns for dsp_solve_segmented
    size_t seg_cap = 0;

    bool has_pulse = false;
    int64_t n_steps = 0, cursor = 0;
    double dt = 0, a_in[2] = {0, 0}, a_out[2] = {0, 0};
    int32_t level = 0;
    double theta_max = 0.0;
    int32_t group = 1;  // FP32_MIXED: steps multiplied per update (choose_group)
    int32_t tdeg = 0;   // FP32_MIXED: tan series degree of the step groups (choose_tan_degree)
    bool withhold_next = false;  // test hook, see dsp_test_withhold_next_copy
    bool fresh = true;      // state not yet written on the device
    bool projected = false;  // partial sums valid for the current pulse
    bool keep_final_state = true;  // dsp_set_keep_final_state
    int32_t tiling = 1;  // test hook dsp_test_tiling: 0 contiguous, 1 automatic, 2 no tail split
    bool state_stale = false;  // the last launch did not write the final state back
    dsp_status latched = DSP_OK;
};

namespace {

bool finite(double x) { return std::isfinite(x); }

dsp_status latch_cuda(dsp_grid *g, cudaError_t e)
{
    if (e == cudaSuccess)
        return DSP_OK;
    if (g && g->latched == DSP_OK)
        g->latched = DSP_E_CUDA;
    return DSP_E_CUDA;
}

size_t map_elem_bytes(int32_t precision) { return precision == DSP_FP64 ? 8 : 4; }

// Lowest series level whose truncation error stays inside a fixed budget over
// the whole run.  Truncating cos(theta) after x^dc leaves dc_err ~ x^(dc+1)/(2dc+2)!,
// truncating sin(theta)/theta after x^ds leaves ds_err ~ x^(ds+1)/(2ds+3)!
// (x = theta^2; alternating series, so the first omitted term bounds the error).
// Both errors have a fixed sign, so they add up over steps: per step they
// perturb the norm by ~2 dc_err + 2 x ds_err and the rotation angle by
// ~theta ds_err.  The budget over n_steps steps is 1e-6 (FP32_MIXED: a tenth of
// its 1e-5 target, and below its own rounding error; on every point of the
// 2048^2 x 1e5-step LZS maps the per-point maxima are the same as with a 2e-8
// budget) or 1e-16 (FP64).
int32_t choose_level(int32_t precision, double theta, int64_t n_steps)
{
    const double x = theta * theta;
    const double budget =
        (precision == DSP_FP64 ? 1e-16 : 1e-6) / static_cast<double>(std::max<int64_t>(n_steps, 1));
    const dsp::SeriesLevel *lv = precision == DSP_FP64 ? dsp::kLevelsF64 : dsp::kLevelsF32;
    for (int i = 0; i < dsp::kNumLevels; ++i) {
        double fc = 1.0, fs = 1.0;  // (2dc+2)!, (2ds+3)!
        for (int k = 2; k <= 2 * lv[i].dc + 2; ++k)
            fc *= k;
        for (int k = 2; k <= 2 * lv[i].ds + 3; ++k)
            fs *= k;
        const double dc_err = std::pow(x, lv[i].dc + 1) / fc;
        const double ds_err = std::pow(x, lv[i].ds + 1) / fs;
        const double err = std::max(2.0 * dc_err + 2.0 * x * ds_err, theta * ds_err);
        if (err <= budget)
            return i;
    }
    return dsp::kNumLevels - 1;
}

// Degree DT of the tan (STRANG_XY: and sec) series of the tan-normalised groups
// (FP32_MIXED, every scheme; MAGNUS4 in x = |n|^2): the lowest of kTanDegrees whose truncation
// stays inside the FP32_MIXED budget over the run.  Dropping x^(DT+1) and beyond
// perturbs the step's rotation angle by ~theta c_(DT+1) x^(DT+1), with a fixed
// sign, so it adds up over the steps.  0: no degree is enough (groups are not used).
int32_t choose_tan_degree(int32_t scheme, double theta, int64_t n_steps)
{
    const double x = theta * theta;
    const double budget = 1e-6 / static_cast<double>(std::max<int64_t>(n_steps, 1));
    for (int i = 0; i < dsp::kNumTanDegrees; ++i) {
        const int d = dsp::kTanDegrees[i];
        const double c = scheme == DSP_SCHEME_STRANG_XY
                             ? std::max(dsp::kTanSeries[d + 1], dsp::kSecSeries[d + 1])
                             : dsp::kTanSeries[d + 1];
        if (theta * c * std::pow(x, d + 1) <= budget)
            return d;
    }
    return 0;
}

// Steps multiplied into one operator before each compensated update (FP32_MIXED,
// every scheme): the largest G in {16, 8, 4, 2} whose group rotation G *
// theta_max stays within the scheme's group angle (kGroupAngleTan for EXACT and
// STRANG_XY, kGroupAngleMagnus for MAGNUS4), else 1.  Groups need a tan degree
// (tdeg > 0).
int32_t choose_group(int32_t precision, int32_t scheme, int32_t tdeg, double theta_max)
{
    if (precision != DSP_FP32_MIXED || tdeg <= 0)
        return 1;
    const double angle =
        scheme == DSP_SCHEME_MAGNUS4 ? dsp::kGroupAngleMagnus : dsp::kGroupAngleTan;
    for (int32_t G = dsp::kGroupMax; G >= 2; G /= 2)
        if (G * theta_max <= angle)
            return G;
    return 1;
}

// dt * max over steps and box corners of |p + A_n| (|P| is convex in p, so the
// maximum over the box is at a corner).  The squared magnitude of a corner is
// (c_x + A_x)^2 + (c_y + A_y)^2, and a rounded sum grows with either term, so
// the largest corner of a step is the larger x square plus the larger y square:
// two squares per coordinate and one square root for the whole table.  If the
// squares overflow (|p + A| above ~1e154), the maximum is taken with hypot.
double theta_max(const dsp_grid *g, const double *a_mid, int64_t n, double dt)
{
    const double cx0 = g->px_min, cx1 = g->px_max, cy0 = g->py_min, cy1 = g->py_max;
    double m2 = 0.0;
    for (int64_t k = 0; k < n; ++k) {
        const double x0 = cx0 + a_mid[2 * k], x1 = cx1 + a_mid[2 * k];
        const double y0 = cy0 + a_mid[2 * k + 1], y1 = cy1 + a_mid[2 * k + 1];
        m2 = std::max(m2, std::max(x0 * x0, x1 * x1) + std::max(y0 * y0, y1 * y1));
    }
    if (std::isfinite(m2))
        return dt * std::sqrt(m2);
    double m = 0.0;
    const double cx[2] = {cx0, cx1}, cy[2] = {cy0, cy1};
    for (int64_t k = 0; k < n; ++k)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                m = std::max(m, std::hypot(cx[i] + a_mid[2 * k], cy[j] + a_mid[2 * k + 1]));
    return dt * m;
}

dsp_status check_usable(const dsp_grid *g)
{
    if (!g)
        return DSP_E_INVALID;
    return g->latched;
}

// Grids whose rows split into whole 256-column strips evolve on row-strip tiles
// (ReqDesc::strips): FP32_MIXED in every scheme, FP64 in EXACT and STRANG_XY.
// Every point's arithmetic is the same on either tiling.
bool use_strips(const dsp_grid *g)
{
    return g->tiling != 0 && g->nx % dsp::kStripWidth == 0 &&
           (g->precision == DSP_FP32_MIXED || g->scheme != DSP_SCHEME_MAGNUS4);
}

int32_t strip_tiles(const dsp_grid *g)
{
    return static_cast<int32_t>((g->nx / dsp::kStripWidth) *
                                ((static_cast<int64_t>(g->ny) + dsp::kStripHeight - 1) /
                                 dsp::kStripHeight));
}

ReqDesc make_desc(const dsp_grid *g, int64_t begin, int64_t end, bool project, void *map)
{
    ReqDesc r;
    std::memset(&r, 0, sizeof(r));
    r.table = g->table;
    r.state = g->state;
    r.map = map;
    r.partials = g->partials;
    r.err = g->scal ? &g->scal->err : nullptr;
    r.nodes_out = g->nodes;
    r.px_min = g->px_min;
    r.py_min = g->py_min;
    r.hx = g->hx;
    r.hy = g->hy;
    r.dt = g->dt;
    r.a_in[0] = g->a_in[0];
    r.a_in[1] = g->a_in[1];
    r.a_out[0] = g->a_out[0];
    r.a_out[1] = g->a_out[1];
    r.n_points = g->n_points;
    r.step_begin = begin;
    r.step_end = end;
    r.nx = g->nx;
    r.ny = g->ny;
    r.row0 = g->row0;
    // A state that is only read (a projection of the state on the device) is not
    // written back; with keep_final_state off, neither is the state after the
    // last step when it is projected in the same launch.
    const bool read_only = begin == end && !g->fresh;
    const bool final_dropped = project && end == g->n_steps && !g->keep_final_state;
    r.store_state = (read_only || final_dropped) ? 0 : 1;
    r.scheme = g->scheme;
    r.valley = g->valley;
    r.level = g->level;
    r.fresh = g->fresh ? 1 : 0;
    r.project = project ? 1 : 0;
    r.n_tiles = g->n_tiles;
    // a projection of the state on the device runs on contiguous tiles
    r.strips = use_strips(g) && !(read_only && project) ? 1 : 0;
    r.strip_h = dsp::kStripHeight;
    r.strip_row0 = 0;
    r.tail_split = g->tiling == 1 ? 1 : 0;
    if (r.strips)
        r.n_tiles = strip_tiles(g);
    r.group = g->group;
    r.tdeg = g->tdeg;
    r.withhold_first_copy = g->withhold_next ? 1 : 0;
    r.table_steps = g->table_cap;
    return r;
}

double density_scale(const dsp_grid *g)
{
    return 4.0 / ((2.0 * kPi) * (2.0 * kPi)) * g->hx * g->hy;
}

// A launch that only projects a state already on the device.
bool project_only(const ReqDesc &r)
{
    return r.step_begin == r.step_end && r.project && !r.fresh && r.nodes_out;
}

// Wave quantisation of a launch of one grid on row strips.  The strip kernel
// holds S = SMs x (CTAs per SM) tiles at once; when the grid's T tiles leave a
// last wave of r = T mod S tiles that is at most half full, the last ceil(r /
// (nx / 256)) 4-row strips are launched instead as twice as many 2-row strips
// (strip_h = 2, the same points at half the work per CTA), so that the last
// wave takes about half as long.  Grids of at most half a wave are all 2-row
// strips.  Every point's arithmetic, and every granule, is unchanged: only
// which CTA computes which rows.  Returns the descriptors to launch.
std::vector<ReqDesc> split_last_wave(const ReqDesc &r, int precision)
{
    std::vector<ReqDesc> out(1, r);
    if (!r.strips || !r.tail_split || r.strip_h != dsp::kStripHeight)
        return out;
    // per kernel: [0] FP64, [1 + scheme] FP32_MIXED; looked up once for the process
    // (handles may be used from different host threads, so under a lock)
    static std::mutex cache_mutex;
    static int sms[4] = {0, 0, 0, 0}, per_sm[4] = {0, 0, 0, 0};
    const int p = precision == DSP_FP64 ? 0 : 1 + r.scheme;
    int n_sm = 0, n_per_sm = 0;
    {
        std::lock_guard<std::mutex> lock(cache_mutex);
        if (sms[p] == 0) {
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&sms[p], cudaDevAttrMultiProcessorCount, dev) !=
                    cudaSuccess ||
                dsp::strip_ctas_per_sm(precision == DSP_FP64 ? 0 : 1, r.scheme, &per_sm[p]) !=
                    cudaSuccess ||
                per_sm[p] < 1) {
                cudaGetLastError();
                sms[p] = -1;
            }
        }
        n_sm = sms[p];
        n_per_sm = per_sm[p];
    }
    if (n_sm <= 0)
        return out;
    const int64_t S = static_cast<int64_t>(n_sm) * n_per_sm;
    const int64_t ncb = r.nx / dsp::kStripWidth;
    const int64_t nstrips = (r.ny + dsp::kStripHeight - 1) / dsp::kStripHeight;
    const int64_t T = ncb * nstrips;
    const int64_t rem = T % S;
    if (rem == 0)
        return out;
    const int64_t k = std::min<int64_t>(nstrips, (rem + ncb - 1) / ncb);  // strips to halve
    const int64_t row_tail = dsp::kStripHeight * (nstrips - k);
    const int64_t tail_tiles = ncb * ((r.ny - row_tail + 1) / 2);
    if (tail_tiles > S)
        return out;
    out.clear();
    if (nstrips > k) {
        ReqDesc full = r;
        full.n_tiles = static_cast<int32_t>(ncb * (nstrips - k));
        out.push_back(full);
    }
    ReqDesc tail = r;
    tail.strip_h = 2;
    tail.strip_row0 = static_cast<int32_t>(row_tail);
    tail.n_tiles = static_cast<int32_t>(tail_tiles);
    out.push_back(tail);
    return out;
}

// Queues launches advancing several requests of one precision.  Requests go to
// their kernel -- FP64 or FP32_MIXED, on contiguous tiles or on row strips, or
// the projection kernel when every request only projects -- and are split into
// launches of at most kMaxReqPerLaunch.  Each request reports device errors in
// its own error word (ReqDesc::err).  A launch of one grid on row strips has its
// last wave split (split_last_wave).
cudaError_t launch_requests(const std::vector<ReqDesc> &reqs, int precision, cudaStream_t stream)
{
    bool proj = !reqs.empty();
    for (const ReqDesc &r : reqs)
        proj = proj && project_only(r);
    std::vector<ReqDesc> split;
    if (!proj && reqs.size() == 1)
        split = split_last_wave(reqs[0], precision);
    const std::vector<ReqDesc> &all = split.empty() ? reqs : split;
    // kernel kinds: 0 contiguous tiles; 1 + 2 scheme + (strip_h == 2): row strips
    const auto kind_of = [&](const ReqDesc &r) {
        return proj || !r.strips ? 0 : 1 + 2 * r.scheme + (r.strip_h == 2 ? 1 : 0);
    };
    for (int kind = 0; kind < 7; ++kind) {
        std::vector<const ReqDesc *> sel;
        for (const ReqDesc &r : all)
            if (kind_of(r) == kind)
                sel.push_back(&r);
        size_t i = 0;
        while (i < sel.size()) {
            std::unique_ptr<EvolveArgs> a(new EvolveArgs());
            std::memset(a.get(), 0, sizeof(EvolveArgs));
            int tiles = 0;
            int n = 0;
            while (i < sel.size() && n < dsp::kMaxReqPerLaunch) {
                a->r[n] = *sel[i];
                a->r[n].tile_begin = tiles;
                tiles += sel[i]->n_tiles;
                ++n;
                ++i;
            }
            a->nreq = n;
            a->total_tiles = tiles;
            cudaError_t e;
            if (proj)
                e = dsp::launch_project(*a, precision, stream);
            else if (precision == DSP_FP64)
                e = kind == 0 ? dsp::launch_evolve_f64(*a, stream)
                              : dsp::launch_evolve_f64_strip(*a, stream);
            else if (kind == 0)
                e = dsp::launch_evolve_mixed(*a, stream);
            else
                e = dsp::launch_evolve_strip(*a, (kind - 1) / 2, (kind - 1) % 2 ? 2 : 4, stream);
            if (e != cudaSuccess)
                return e;
        }
    }
    return cudaSuccess;
}

cudaError_t launch_finalizes(const std::vector<dsp::FinDesc> &fins, cudaStream_t stream)
{
    size_t i = 0;
    while (i < fins.size()) {
        FinalizeArgs a;
        std::memset(&a, 0, sizeof(a));
        int n = 0;
        while (i < fins.size() && n < dsp::kMaxFinPerLaunch)
            a.f[n++] = fins[i++];
        a.count = n;
        cudaError_t e = dsp::launch_finalize(a, stream);
        if (e != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

dsp::FinDesc fin_desc(const dsp_grid *g)
{
    dsp::FinDesc f;
    std::memset(&f, 0, sizeof(f));
    f.partials = g->partials;
    f.n_parts = g->n_parts;
    f.scale = density_scale(g);
    f.out = &g->scal->density;
    return f;
}

// Reads the device scalars after the stream has drained.
dsp_status read_scalars(dsp_grid *g, double *density)
{
    DeviceScalars h;
    cudaError_t e = cudaMemcpyAsync(&h, g->scal, sizeof(h), cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess)
        return latch_cuda(g, e);
    if (h.err & dsp::kErrTimeout) {
        g->latched = DSP_E_TIMEOUT;
        return DSP_E_TIMEOUT;
    }
    if (h.err & dsp::kErrBounds) {
        g->latched = DSP_E_BOUNDS;
        return DSP_E_BOUNDS;
    }
    if (density)
        *density = h.density;
    return DSP_OK;
}

dsp_status validate_grid_args(int32_t nx, int32_t ny, double px_min, double px_max,
                              double py_min, double py_max, int32_t precision, int32_t scheme,
                              int32_t valley)
{
    if (nx < 1 || ny < 1 || static_cast<int64_t>(nx) * ny > 2147483647LL)
        return DSP_E_INVALID;
    if (!finite(px_min) || !finite(px_max) || !finite(py_min) || !finite(py_max))
        return DSP_E_INVALID;
    if (!(px_min < px_max) || !(py_min < py_max))
        return DSP_E_INVALID;
    if (precision != DSP_FP64 && precision != DSP_FP32_MIXED)
        return DSP_E_INVALID;
    if (scheme != DSP_SCHEME_EXACT && scheme != DSP_SCHEME_STRANG_XY &&
        scheme != DSP_SCHEME_MAGNUS4)
        return DSP_E_INVALID;
    if (valley != 1 && valley != -1)
        return DSP_E_INVALID;
    return DSP_OK;
}

// Checks a pulse's arguments (and its step condition); *tmax_out, when given,
// receives theta_max of the table (0 for an empty one).
dsp_status validate_pulse_args(const dsp_grid *g, const double *a_mid, int64_t n_steps, double dt,
                               const double a_in[2], const double a_out[2],
                               double *tmax_out = nullptr)
{
    if (n_steps < 0 || (n_steps > 0 && !a_mid) || !a_in || !a_out)
        return DSP_E_INVALID;
    if (!finite(dt) || dt < 0.0 || (n_steps > 0 && !(dt > 0.0)))
        return DSP_E_INVALID;
    if (!finite(a_in[0]) || !finite(a_in[1]) || !finite(a_out[0]) || !finite(a_out[1]))
        return DSP_E_INVALID;
    for (int64_t k = 0; k < 2 * n_steps; ++k)
        if (!finite(a_mid[k]))
            return DSP_E_INVALID;
    const double tmax = n_steps > 0 ? theta_max(g, a_mid, n_steps, dt) : 0.0;
    if (tmax > kPi)
        return DSP_E_CFL;
    if (tmax_out)
        *tmax_out = tmax;
    return DSP_OK;
}

// A(t) samples per step in the caller's table: one (A_x, A_y) at the midpoint,
// or two (at the Gauss points) for MAGNUS4.
int samples_per_step(int32_t scheme) { return scheme == DSP_SCHEME_MAGNUS4 ? 2 : 1; }

// Bytes per step of the device table: per A sample, double2 (FP64) or float2
// (FP32_MIXED).
size_t entry_bytes(int32_t precision, int32_t scheme)
{
    return (precision == DSP_FP64 ? 16 : 8) * static_cast<size_t>(samples_per_step(scheme));
}

// Device bytes of a table of n steps: padded to 16 bytes, because the kernels
// stage it with 1-D bulk copies that start and end on 16-byte boundaries.
size_t table_bytes(int32_t precision, int32_t scheme, int64_t n)
{
    return (entry_bytes(precision, scheme) * static_cast<size_t>(n) + 15) & ~static_cast<size_t>(15);
}

// Fills the table layout the kernels read (see ReqDesc::table).
void build_table(const dsp_grid *g, const double *a_mid, int64_t n, double dt,
                 std::vector<unsigned char> &out)
{
    out.resize(static_cast<size_t>(n) * entry_bytes(g->precision, g->scheme));
    // valley K- is stepped as K+ on -P, so its table holds -dt*A
    const double vs = g->valley > 0 ? 1.0 : -1.0;
    if (g->scheme == DSP_SCHEME_MAGNUS4) {
        // (Abar, D): Abar = (A1 + A2)/2, D = -(sqrt(3)/6) (A2 - A1), both times s*dt
        const double kappa = -std::sqrt(3.0) / 6.0;
        double mresid[2] = {0.0, 0.0};
        for (int64_t k = 0; k < n; ++k) {
            const double *a = a_mid + 4 * k;
            const double bx = vs * (dt * (0.5 * (a[0] + a[2])));
            const double by = vs * (dt * (0.5 * (a[1] + a[3])));
            const double dx = kappa * (vs * (dt * (a[2] - a[0])));
            const double dy = kappa * (vs * (dt * (a[3] - a[1])));
            if (g->precision == DSP_FP64) {
                double *t = reinterpret_cast<double *>(out.data()) + 4 * k;
                t[0] = bx;
                t[1] = by;
                t[2] = dx;
                t[3] = dy;
            } else {
                // Abar rounded with error feedback, as for the midpoint table below
                float *t = reinterpret_cast<float *>(out.data()) + 4 * k;
                const double vx = bx + mresid[0], vy = by + mresid[1];
                t[0] = static_cast<float>(vx);
                t[1] = static_cast<float>(vy);
                mresid[0] = vx - static_cast<double>(t[0]);
                mresid[1] = vy - static_cast<double>(t[1]);
                t[2] = static_cast<float>(dx);
                t[3] = static_cast<float>(dy);
            }
        }
        return;
    }
    if (g->precision == DSP_FP64) {
        double *t = reinterpret_cast<double *>(out.data());
        for (int64_t k = 0; k < n; ++k) {
            t[2 * k] = vs * (dt * a_mid[2 * k]);
            t[2 * k + 1] = vs * (dt * a_mid[2 * k + 1]);
        }
    } else {
        // Rounded with error feedback: each entry absorbs the previous entries'
        // rounding residual, so the running sum of the stored dt*A stays within half
        // a float ulp of the exact running sum.  The phase integrates A over time; the
        // per-step roundings then cannot random-walk in it, however long the run.
        float *t = reinterpret_cast<float *>(out.data());
        double resid[2] = {0.0, 0.0};
        for (int64_t k = 0; k < n; ++k)
            for (int c = 0; c < 2; ++c) {
                const double v = vs * (dt * a_mid[2 * k + c]) + resid[c];
                const float f = static_cast<float>(v);
                resid[c] = v - static_cast<double>(f);
                t[2 * k + c] = f;
            }
    }
}

// Projection nodes of the grid's columns and rows, s (p + A_out) with s the
// valley, formed in FP64 as the kernels form the grid nodes (p = lo + (i + 1/2) h),
// each split into an FP32 hi + lo pair for the double-float projection: nx
// columns, then the grid's ny rows (global rows row0 ...).
void build_nodes(const dsp_grid *g, std::vector<float2> &out)
{
    out.resize(static_cast<size_t>(g->nx) + static_cast<size_t>(g->ny));
    const double vs = g->valley > 0 ? 1.0 : -1.0;
    const auto put = [&](size_t k, double v) {
        const float h = static_cast<float>(v);
        out[k] = make_float2(h, static_cast<float>(v - static_cast<double>(h)));
    };
    for (int32_t i = 0; i < g->nx; ++i) {
        const double p = g->px_min + (static_cast<double>(i) + 0.5) * g->hx;
        put(static_cast<size_t>(i), vs * (p + g->a_out[0]));
    }
    for (int32_t j = 0; j < g->ny; ++j) {
        const double p = g->py_min + (static_cast<double>(g->row0 + j) + 0.5) * g->hy;
        put(static_cast<size_t>(g->nx) + static_cast<size_t>(j), vs * (p + g->a_out[1]));
    }
}

size_t node_bytes(const dsp_grid *g)
{
    return sizeof(float2) * (static_cast<size_t>(g->nx) + static_cast<size_t>(g->ny));
}

void free_grid_memory(dsp_grid *g)
{
    if (g->owns_state && g->state)
        cudaFree(g->state);
    if (g->table)
        cudaFree(g->table);
    if (g->partials)
        cudaFree(g->partials);
    if (g->scal)
        cudaFree(g->scal);
    if (g->own_map)
        cudaFree(g->own_map);
    if (g->nodes)
        cudaFree(g->nodes);
    if (g->seg_buf)
        cudaFree(g->seg_buf);
    g->seg_buf = nullptr;
    g->seg_cap = 0;
    g->state = g->table = g->own_map = nullptr;
    g->partials = nullptr;
    g->scal = nullptr;
    g->nodes = nullptr;
}

// Geometry and arithmetic fields of a grid (no allocation): rows [row0, row0 +
// rows) of the nx by ny grid on the box.
void fill_grid(dsp_grid *g, int32_t nx, int32_t ny, double px_min, double px_max, double py_min,
               double py_max, int32_t precision, int32_t scheme, int32_t valley,
               cudaStream_t stream, int32_t row0 = 0, int32_t rows = -1)
{
    if (rows < 0)
        rows = ny;
    g->nx = nx;
    g->ny = rows;
    g->row0 = row0;
    g->ny_total = ny;
    g->precision = precision;
    g->scheme = scheme;
    g->valley = valley;
    g->px_min = px_min;
    g->px_max = px_max;
    g->py_min = py_min;
    g->py_max = py_max;
    g->hx = (px_max - px_min) / nx;
    g->hy = (py_max - py_min) / ny;
    g->n_points = static_cast<int64_t>(nx) * rows;
    g->n_tiles = static_cast<int32_t>((g->n_points + dsp::kTilePoints - 1) / dsp::kTilePoints);
    g->n_parts = (g->n_points + dsp::kGranule - 1) / dsp::kGranule;
    g->stream = stream;
}

dsp_status create_grid_impl(int32_t nx, int32_t ny, double px_min, double px_max, double py_min,
                            double py_max, int32_t precision, int32_t scheme, int32_t valley,
                            cudaStream_t stream, void *state_dev, int64_t state_bytes,
                            dsp_grid **out, int32_t row_begin = 0, int32_t row_end = -1)
{
    if (!out)
        return DSP_E_INVALID;
    *out = nullptr;
    if (row_end < 0)
        row_end = ny;
    if (ny < 1 || row_begin < 0 || row_begin >= row_end || row_end > ny)
        return DSP_E_INVALID;
    // the grid holds nx x (row_end - row_begin) points; ny only sets the spacing
    dsp_status s = validate_grid_args(nx, row_end - row_begin, px_min, px_max, py_min, py_max,
                                      precision, scheme, valley);
    if (s != DSP_OK)
        return s;
    const int64_t need = dsp_state_bytes(nx, row_end - row_begin, precision);
    if (state_dev && (state_bytes < need || (reinterpret_cast<uintptr_t>(state_dev) & 15u)))
        return DSP_E_INVALID;
    dsp_grid *g = new (std::nothrow) dsp_grid();
    if (!g)
        return DSP_E_NOMEM;
    fill_grid(g, nx, ny, px_min, px_max, py_min, py_max, precision, scheme, valley, stream,
              row_begin, row_end - row_begin);
    cudaError_t e = cudaSuccess;
    if (state_dev) {
        g->state = state_dev;
    } else {
        e = cudaMalloc(&g->state, static_cast<size_t>(need));
        g->owns_state = (e == cudaSuccess);
    }
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&g->partials),
                       sizeof(double) * static_cast<size_t>(g->n_parts));
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&g->scal), sizeof(DeviceScalars));
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&g->nodes), node_bytes(g));
    if (e == cudaSuccess)
        e = cudaMemsetAsync(g->scal, 0, sizeof(DeviceScalars), stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_grid_memory(g);
        delete g;
        return e == cudaErrorMemoryAllocation ? DSP_E_NOMEM : DSP_E_CUDA;
    }
    *out = g;
    return DSP_OK;
}

// Host part of setting a pulse: validates, fills the grid's pulse fields, lays
// out the device table in `host` and the projection nodes in `nodes`.  Nothing
// is queued.
dsp_status prepare_pulse(dsp_grid *g, const double *a_mid, int64_t n_steps, double dt,
                         const double a_in[2], const double a_out[2],
                         std::vector<unsigned char> &host, std::vector<float2> &nodes)
{
    // every (A_x, A_y) sample of the table, whatever the samples per step
    const int64_t n_samples = n_steps * samples_per_step(g->scheme);
    double tmax = 0.0;
    dsp_status s = validate_pulse_args(g, a_mid, n_samples, dt, a_in, a_out, &tmax);
    if (s != DSP_OK)
        return s;
    build_table(g, a_mid, n_steps, dt, host);
    g->has_pulse = true;
    g->n_steps = n_steps;
    g->cursor = 0;
    g->dt = dt;
    g->a_in[0] = a_in[0];
    g->a_in[1] = a_in[1];
    g->a_out[0] = a_out[0];
    g->a_out[1] = a_out[1];
    g->theta_max = tmax;
    g->level = choose_level(g->precision, tmax, n_steps);
    g->tdeg = g->precision == DSP_FP32_MIXED ? choose_tan_degree(g->scheme, tmax, n_steps) : 0;
    g->group = choose_group(g->precision, g->scheme, g->tdeg, tmax);
    g->fresh = true;
    g->projected = false;
    g->state_stale = false;
    build_nodes(g, nodes);
    return DSP_OK;
}

dsp_status set_pulse_impl(dsp_grid *g, const double *a_mid, int64_t n_steps, double dt,
                          const double a_in[2], const double a_out[2])
{
    dsp_grid staged = *g;
    std::vector<unsigned char> host;
    std::vector<float2> nodes;
    dsp_status s = prepare_pulse(&staged, a_mid, n_steps, dt, a_in, a_out, host, nodes);
    if (s != DSP_OK)
        return s;
    cudaError_t e = cudaSuccess;
    if (n_steps > g->table_cap) {
        if (g->table) {
            e = cudaStreamSynchronize(g->stream);  // old table may still be read
            if (e == cudaSuccess)
                e = cudaFree(g->table);
            g->table = nullptr;
            g->table_cap = 0;
        }
        if (e == cudaSuccess)
            e = cudaMalloc(&g->table, table_bytes(g->precision, g->scheme, n_steps));
        if (e != cudaSuccess) {
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? DSP_E_NOMEM : latch_cuda(g, e);
        }
        g->table_cap = n_steps;
    }
    if (n_steps > 0) {
        e = cudaMemcpyAsync(g->table, host.data(), host.size(), cudaMemcpyHostToDevice, g->stream);
        if (e != cudaSuccess)
            return latch_cuda(g, e);
    }
    e = cudaMemcpyAsync(g->nodes, nodes.data(), node_bytes(g), cudaMemcpyHostToDevice, g->stream);
    if (e != cudaSuccess)
        return latch_cuda(g, e);
    staged.table = g->table;
    staged.table_cap = g->table_cap;
    *g = staged;
    return DSP_OK;
}

// Advances one grid to `end`, optionally projecting into `map` at the end.
dsp_status run_one(dsp_grid *g, int64_t end, bool project, void *map)
{
    if (g->state_stale && !g->fresh)
        return DSP_E_STATE;  // the final state was not kept (dsp_set_keep_final_state)
    std::vector<ReqDesc> r(1, make_desc(g, g->cursor, end, project, map));
    g->withhold_next = false;
    cudaError_t e = launch_requests(r, g->precision, g->stream);
    if (e != cudaSuccess)
        return latch_cuda(g, e);
    if (!r[0].store_state && !(r[0].step_begin == r[0].step_end && !r[0].fresh))
        g->state_stale = true;
    g->cursor = end;
    g->fresh = false;
    if (project)
        g->projected = true;
    return DSP_OK;
}

dsp_status ensure_own_map(dsp_grid *g)
{
    if (g->own_map)
        return DSP_OK;
    cudaError_t e =
        cudaMalloc(&g->own_map, static_cast<size_t>(g->n_points) * map_elem_bytes(g->precision));
    if (e != cudaSuccess) {
        cudaGetLastError();
        g->own_map = nullptr;
        return DSP_E_NOMEM;
    }
    return DSP_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

int64_t dsp_state_bytes(int32_t nx, int32_t ny, int32_t precision)
{
    if (nx < 1 || ny < 1 || static_cast<int64_t>(nx) * ny > 2147483647LL)
        return -1;
    if (precision != DSP_FP64 && precision != DSP_FP32_MIXED)
        return -1;
    return 32 * static_cast<int64_t>(nx) * ny;
}

dsp_status dsp_create_grid(int32_t nx, int32_t ny, double px_min, double px_max, double py_min,
                           double py_max, int32_t precision, int32_t scheme, int32_t valley,
                           void *cuda_stream, void *state_dev, int64_t state_dev_bytes,
                           dsp_grid **out)
{
    return create_grid_impl(nx, ny, px_min, px_max, py_min, py_max, precision, scheme, valley,
                            static_cast<cudaStream_t>(cuda_stream), state_dev, state_dev_bytes,
                            out);
}

dsp_status dsp_create_band(int32_t nx, int32_t ny, int32_t row_begin, int32_t row_end,
                           double px_min, double px_max, double py_min, double py_max,
                           int32_t precision, int32_t scheme, int32_t valley, void *cuda_stream,
                           void *state_dev, int64_t state_dev_bytes, dsp_grid **out)
{
    if (out)
        *out = nullptr;
    if (row_end < 0)
        return DSP_E_INVALID;
    return create_grid_impl(nx, ny, px_min, px_max, py_min, py_max, precision, scheme, valley,
                            static_cast<cudaStream_t>(cuda_stream), state_dev, state_dev_bytes,
                            out, row_begin, row_end);
}

dsp_status dsp_set_keep_final_state(dsp_grid *g, int32_t keep)
{
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    if (keep != 0 && keep != 1)
        return DSP_E_INVALID;
    g->keep_final_state = keep != 0;
    return DSP_OK;
}

dsp_status dsp_set_pulse(dsp_grid *g, const double *a_mid, int64_t n_steps, double dt,
                         const double a_in[2], const double a_out[2])
{
    Range range_("dsp_set_pulse");
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    return set_pulse_impl(g, a_mid, n_steps, dt, a_in, a_out);
}

dsp_status dsp_evolve(dsp_grid *g, int64_t steps)
{
    Range range_("dsp_evolve");
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    if (steps < 0)
        return DSP_E_INVALID;
    if (!g->has_pulse || g->cursor + steps > g->n_steps)
        return DSP_E_STATE;
    if (steps == 0)
        return DSP_OK;
    g->projected = false;
    return run_one(g, g->cursor + steps, false, nullptr);
}

dsp_status dsp_project(dsp_grid *g, void *map_dev)
{
    Range range_("dsp_project");
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    if (!map_dev)
        return DSP_E_INVALID;
    if (!g->has_pulse || g->cursor != g->n_steps)
        return DSP_E_STATE;
    return run_one(g, g->cursor, true, map_dev);
}

dsp_status dsp_reduce_density(dsp_grid *g, double *n_host)
{
    Range range_("dsp_reduce_density");
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    if (!n_host)
        return DSP_E_INVALID;
    if (!g->projected)
        return DSP_E_STATE;
    std::vector<dsp::FinDesc> f(1, fin_desc(g));
    cudaError_t e = launch_finalizes(f, g->stream);
    if (e != cudaSuccess)
        return latch_cuda(g, e);
    return read_scalars(g, n_host);
}

dsp_status dsp_solve(dsp_grid *g, void *map_dev, double *n_host)
{
    Range range_("dsp_solve");
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    if (!g->has_pulse)
        return DSP_E_STATE;
    if (!map_dev) {
        s = ensure_own_map(g);
        if (s != DSP_OK)
            return s;
        map_dev = g->own_map;
    }
    s = run_one(g, g->n_steps, true, map_dev);
    if (s != DSP_OK)
        return s;
    std::vector<dsp::FinDesc> f(1, fin_desc(g));
    cudaError_t e = launch_finalizes(f, g->stream);
    if (e != cudaSuccess)
        return latch_cuda(g, e);
    if (n_host)
        return read_scalars(g, n_host);
    return DSP_OK;
}

dsp_status dsp_solve_segmented(dsp_grid *g, int32_t segments, void *map_dev, double *n_host)
{
    Range range_("dsp_solve_segmented");
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    if (segments < 0)
        return DSP_E_INVALID;
    if (!g->has_pulse || g->cursor != 0)
        return DSP_E_STATE;
    if (g->n_steps == 0)
        return dsp_solve(g, map_dev, n_host);
    int64_t S = segments;
    if (S == 0) {
        // FP64 evolution is bound by the FP64 pipe: one segment-tile per SM.  FP32_MIXED
        // segments are short and latency bound, and the FP64 combine grows with S: one
        // segment-tile per two SMs.  At least 16 steps a segment.  (Measured on the 64^2
        // x 2000-step case, 4 tiles: S = 38 / 19 beat S = 76 by 8% / 40%.)
        // looked up once for the process (a thread-safe static initialisation)
        static const int sms = [] {
            int dev = 0, n = 0;
            if (cudaGetDevice(&dev) != cudaSuccess ||
                cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
                n < 1) {
                cudaGetLastError();
                return 152;
            }
            return n;
        }();
        const int64_t ctas = g->precision == DSP_FP64 ? sms : (sms + 1) / 2;
        S = (ctas + g->n_tiles - 1) / g->n_tiles;
        S = std::min<int64_t>(S, g->n_steps / 16);
    }
    S = std::max<int64_t>(1, std::min<int64_t>(S, g->n_steps));
    const size_t slab = 32 * static_cast<size_t>(g->n_points);
    if (S > 65536 || static_cast<double>(S) * static_cast<double>(slab) > 16.0e9)
        return DSP_E_INVALID;  // segment columns above 16 GB
    const size_t need = static_cast<size_t>(S) * slab;
    cudaError_t e = cudaSuccess;
    if (need > g->seg_cap) {
        if (g->seg_buf) {
            e = cudaStreamSynchronize(g->stream);
            if (e == cudaSuccess)
                e = cudaFree(g->seg_buf);
            g->seg_buf = nullptr;
            g->seg_cap = 0;
        }
        if (e == cudaSuccess)
            e = cudaMalloc(&g->seg_buf, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            g->seg_buf = nullptr;
            return e == cudaErrorMemoryAllocation ? DSP_E_NOMEM : latch_cuda(g, e);
        }
        g->seg_cap = need;
    }
    if (!map_dev) {
        s = ensure_own_map(g);
        if (s != DSP_OK)
            return s;
        map_dev = g->own_map;
    }
    // 1. every segment's operator product, as its first column, in one batched pass
    std::vector<ReqDesc> descs;
    descs.reserve(static_cast<size_t>(S));
    for (int64_t k = 0; k < S; ++k) {
        const int64_t b = k * g->n_steps / S, e_ = (k + 1) * g->n_steps / S;
        ReqDesc d = make_desc(g, b, e_, false, nullptr);
        d.state = static_cast<unsigned char *>(g->seg_buf) + static_cast<size_t>(k) * slab;
        d.fresh = 1;
        d.init_identity = 1;
        descs.push_back(d);
    }
    e = launch_requests(descs, g->precision, g->stream);
    // 2. psi = M_{S-1} ... M_0 v(p + A_in)
    if (e == cudaSuccess) {
        dsp::CombineArgs c;
        std::memset(&c, 0, sizeof(c));
        c.segs = g->seg_buf;
        c.state = g->state;
        c.n_points = g->n_points;
        c.n_segments = static_cast<int32_t>(S);
        c.nx = g->nx;
        c.px_min = g->px_min;
        c.py_min = g->py_min;
        c.hx = g->hx;
        c.hy = g->hy;
        c.a_in[0] = g->a_in[0];
        c.a_in[1] = g->a_in[1];
        c.valley = g->valley;
        c.row0 = g->row0;
        e = dsp::launch_combine(c, g->precision, g->stream);
    }
    if (e != cudaSuccess)
        return latch_cuda(g, e);
    g->fresh = false;
    g->cursor = g->n_steps;
    // 3. projection + tile sums (a zero-step launch), then the density
    s = run_one(g, g->n_steps, true, map_dev);
    if (s != DSP_OK)
        return s;
    std::vector<dsp::FinDesc> f(1, fin_desc(g));
    e = launch_finalizes(f, g->stream);
    if (e != cudaSuccess)
        return latch_cuda(g, e);
    if (n_host)
        return read_scalars(g, n_host);
    return DSP_OK;
}

dsp_status dsp_solve_host(dsp_grid *g, const double *a_mid, int64_t n_steps, double dt,
                          const double a_in[2], const double a_out[2], void *map_host,
                          double *n_host)
{
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    if (!n_host)
        return DSP_E_INVALID;
    s = set_pulse_impl(g, a_mid, n_steps, dt, a_in, a_out);
    if (s != DSP_OK)
        return s;
    s = ensure_own_map(g);
    if (s != DSP_OK)
        return s;
    s = dsp_solve(g, g->own_map, nullptr);
    if (s != DSP_OK)
        return s;
    if (map_host) {
        cudaError_t e =
            cudaMemcpyAsync(map_host, g->own_map,
                            static_cast<size_t>(g->n_points) * map_elem_bytes(g->precision),
                            cudaMemcpyDeviceToHost, g->stream);
        if (e != cudaSuccess)
            return latch_cuda(g, e);
    }
    return read_scalars(g, n_host);
}

dsp_status dsp_evolve_batch(dsp_grid *const *grids, const int64_t *steps, int32_t count)
{
    Range range_("dsp_evolve_batch");
    if (count < 0 || (count > 0 && (!grids || !steps)))
        return DSP_E_INVALID;
    if (count == 0)
        return DSP_OK;
    for (int32_t i = 0; i < count; ++i) {
        dsp_status s = check_usable(grids[i]);
        if (s != DSP_OK)
            return s;
        if (grids[i]->stream != grids[0]->stream || steps[i] < 0)
            return DSP_E_INVALID;
        for (int32_t j = 0; j < i; ++j)
            if (grids[j] == grids[i])
                return DSP_E_INVALID;
        if (!grids[i]->has_pulse || grids[i]->cursor + steps[i] > grids[i]->n_steps)
            return DSP_E_STATE;
    }
    for (int prec = 0; prec < 2; ++prec) {
        std::vector<ReqDesc> reqs;
        for (int32_t i = 0; i < count; ++i) {
            dsp_grid *g = grids[i];
            if (g->precision != prec || steps[i] == 0)
                continue;
            reqs.push_back(make_desc(g, g->cursor, g->cursor + steps[i], false, nullptr));
        }
        if (reqs.empty())
            continue;
        // every descriptor carries its own grid's error word: a timeout or a bounds
        // hit in one grid's tiles is latched on that grid
        cudaError_t e = launch_requests(reqs, prec, grids[0]->stream);
        if (e != cudaSuccess) {
            for (int32_t i = 0; i < count; ++i)
                latch_cuda(grids[i], e);
            return DSP_E_CUDA;
        }
    }
    for (int32_t i = 0; i < count; ++i) {
        if (steps[i] == 0)
            continue;
        grids[i]->withhold_next = false;
        grids[i]->cursor += steps[i];
        grids[i]->fresh = false;
        grids[i]->projected = false;
    }
    return DSP_OK;
}

dsp_status dsp_get_cursor(const dsp_grid *g, int64_t *cursor, int64_t *n_steps)
{
    if (!g || !cursor || !n_steps)
        return DSP_E_INVALID;
    *cursor = g->cursor;
    *n_steps = g->n_steps;
    return DSP_OK;
}

dsp_status dsp_test_withhold_next_copy(dsp_grid *g)
{
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    g->withhold_next = true;
    return DSP_OK;
}

dsp_status dsp_test_tiling(dsp_grid *g, int32_t tiling)
{
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    if (tiling < 0 || tiling > 2)
        return DSP_E_INVALID;
    g->tiling = tiling;
    return DSP_OK;
}

dsp_status dsp_get_info(const dsp_grid *g, dsp_grid_info *info)
{
    if (!g || !info)
        return DSP_E_INVALID;
    std::memset(info, 0, sizeof(*info));
    info->nx = g->nx;
    info->ny = g->ny;
    info->precision = g->precision;
    info->scheme = g->scheme;
    info->valley = g->valley;
    const dsp::SeriesLevel lv =
        (g->precision == DSP_FP64 ? dsp::kLevelsF64 : dsp::kLevelsF32)[g->level];
    info->cos_degree = lv.dc;
    info->sinc_degree = lv.ds;
    info->n_steps = g->n_steps;
    info->cursor = g->cursor;
    info->n_tiles = use_strips(g) ? strip_tiles(g) : g->n_tiles;
    info->group_steps = g->group;
    info->dt = g->dt;
    info->theta_max = g->theta_max;
    info->row_begin = g->row0;
    info->ny_total = g->ny_total;
    info->row_strips = use_strips(g) ? 1 : 0;
    info->tan_degree = g->group > 1 ? g->tdeg : 0;
    return DSP_OK;
}

dsp_status dsp_save_state(dsp_grid *g, void *host_buf, int64_t bytes, int64_t *cursor)
{
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    const int64_t need = dsp_state_bytes(g->nx, g->ny, g->precision);
    if (!host_buf || !cursor || bytes < need)
        return DSP_E_INVALID;
    if (!g->has_pulse || (g->state_stale && !g->fresh))
        return DSP_E_STATE;
    if (g->fresh) {  // materialise v(p + A_in) on the device first
        s = run_one(g, g->cursor, false, nullptr);
        if (s != DSP_OK)
            return s;
    }
    cudaError_t e = cudaMemcpyAsync(host_buf, g->state, static_cast<size_t>(need),
                                    cudaMemcpyDeviceToHost, g->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess)
        return latch_cuda(g, e);
    *cursor = g->cursor;
    return DSP_OK;
}

dsp_status dsp_load_state(dsp_grid *g, const void *host_buf, int64_t bytes, int64_t cursor)
{
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    const int64_t need = dsp_state_bytes(g->nx, g->ny, g->precision);
    if (!host_buf || bytes < need)
        return DSP_E_INVALID;
    if (!g->has_pulse || cursor < 0 || cursor > g->n_steps)
        return DSP_E_STATE;
    cudaError_t e = cudaMemcpyAsync(g->state, host_buf, static_cast<size_t>(need),
                                    cudaMemcpyHostToDevice, g->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(g->stream);
    if (e != cudaSuccess)
        return latch_cuda(g, e);
    g->cursor = cursor;
    g->fresh = false;
    g->projected = false;
    g->state_stale = false;
    return DSP_OK;
}

dsp_status dsp_destroy_grid(dsp_grid *g)
{
    if (!g)
        return DSP_OK;
    if (g->latched != DSP_E_CUDA)
        cudaStreamSynchronize(g->stream);
    free_grid_memory(g);
    delete g;
    return DSP_OK;
}

const char *dsp_status_string(dsp_status s)
{
    switch (s) {
    case DSP_OK: return "ok";
    case DSP_E_INVALID: return "invalid argument";
    case DSP_E_NOMEM: return "out of memory or over budget";
    case DSP_E_CUDA: return "CUDA error";
    case DSP_E_STATE: return "call out of order";
    case DSP_E_CFL: return "time step too large: dt * max|p + A| > pi";
    case DSP_E_TIMEOUT: return "device-side wait timed out";
    case DSP_E_BOUNDS: return "out-of-range index found by a bounds-check build";
    default: return "unknown status";
    }
}

// ===========================================================================
// Pulse sampler
// ===========================================================================

}  // extern "C"

namespace {

// int_a^b cos(w t + ph) dt = (b - a) cos(w (a + b)/2 + ph) sinc(w (b - a)/2),
// the difference of sines written as a product (no cancellation as w -> 0).
double int_cos(double a, double b, double w, double ph)
{
    const double z = 0.5 * w * (b - a);
    const double sinc = z == 0.0 ? 1.0 : std::sin(z) / z;
    return (b - a) * std::cos(0.5 * w * (a + b) + ph) * sinc;
}

// A_x(t) = -int_0^t E_x for the Sec. IV field, in closed form: the sin^2 and
// cos^2 envelopes are written as sums of cosines and integrated exactly.
double paper_ax(const dsp_pulse_spec &s, double t)
{
    const double tr = kPi / (2.0 * s.Omega_rise);
    const double tf = s.T - kPi / (2.0 * s.Omega_fall);
    const double w = s.omega, ph = s.phi;
    t = std::min(std::max(t, 0.0), s.T);
    double acc = 0.0;
    // rise: sin^2(Or t) cos(w t + ph) = cos/2 - cos((w+2Or)t+ph)/4 - cos((w-2Or)t+ph)/4
    {
        const double b = std::min(t, tr);
        if (b > 0.0) {
            const double o2 = 2.0 * s.Omega_rise;
            acc += 0.5 * int_cos(0.0, b, w, ph) - 0.25 * int_cos(0.0, b, w + o2, ph) -
                   0.25 * int_cos(0.0, b, w - o2, ph);
        }
    }
    // flat top
    if (t > tr) {
        const double b = std::min(t, tf);
        if (b > tr)
            acc += int_cos(tr, b, w, ph);
    }
    // fall: cos^2(Of (t - tf)) cos(w t + ph)
    //     = cos/2 + cos((w+2Of)t + ph - 2 Of tf)/4 + cos((w-2Of)t + ph + 2 Of tf)/4
    if (t > tf) {
        const double o2 = 2.0 * s.Omega_fall;
        acc += 0.5 * int_cos(tf, t, w, ph) + 0.25 * int_cos(tf, t, w + o2, ph - o2 * tf) +
               0.25 * int_cos(tf, t, w - o2, ph + o2 * tf);
    }
    return -s.E0 * acc;
}

void pulse_at(const dsp_pulse_spec &s, double t, double *A)
{
    A[0] = 0.0;
    A[1] = 0.0;
    switch (s.kind) {
    case DSP_PULSE_ZERO:
        break;
    case DSP_PULSE_SIN2: {
        const double e = std::sin(kPi * t / s.T);
        const double f = (s.E0 / s.omega) * e * e;
        A[0] = f * std::sin(s.omega * t);
        A[1] = f * s.eps * std::cos(s.omega * t);
        break;
    }
    case DSP_PULSE_GAUSS: {
        const double u = (t - s.t0) / s.tau;
        const double f = (s.E0 / s.omega) * std::exp(-u * u);
        A[0] = f * std::sin(s.omega * t);
        A[1] = f * s.eps * std::cos(s.omega * t);
        break;
    }
    case DSP_PULSE_TWO_COLOUR: {
        const double e = std::sin(kPi * t / s.T);
        const double env = e * e;
        double ax = 0.0, ay = 0.0;
        for (int k = 1; k <= 2; ++k) {
            const double wk = k * s.omega, phk = k == 1 ? 0.0 : s.phase2;
            ax += (s.E0 / wk) * std::sin(wk * t + phk);
            ay += (s.E0 / wk) * std::cos(wk * t + phk);
        }
        A[0] = env * ax;
        A[1] = env * s.eps * ay;
        break;
    }
    case DSP_PULSE_CONST_FIELD:
        A[0] = -s.E0 * (t - 0.5 * s.T);
        break;
    case DSP_PULSE_PAPER:
        A[0] = paper_ax(s, t);
        break;
    default:
        break;
    }
}

bool spec_ok(const dsp_pulse_spec &s)
{
    const double v[] = {s.E0, s.omega, s.T, s.tau, s.t0, s.eps, s.phase2, s.Omega_rise,
                        s.Omega_fall, s.phi};
    for (double x : v)
        if (!std::isfinite(x))
            return false;
    if (!(s.T > 0.0))
        return false;
    switch (s.kind) {
    case DSP_PULSE_ZERO:
    case DSP_PULSE_CONST_FIELD:
        return true;
    case DSP_PULSE_SIN2:
    case DSP_PULSE_TWO_COLOUR:
        return s.omega > 0.0;
    case DSP_PULSE_GAUSS:
        return s.omega > 0.0 && s.tau > 0.0;
    case DSP_PULSE_PAPER:
        return s.omega > 0.0 && s.Omega_rise > 0.0 && s.Omega_fall > 0.0 &&
               kPi / (2.0 * s.Omega_rise) <= s.T - kPi / (2.0 * s.Omega_fall);
    default:
        return false;
    }
}

}  // namespace

extern "C" dsp_status dsp_sample_pulse_gauss(const dsp_pulse_spec *spec, int64_t n_steps,
                                             double *a_gauss, double *a_in, double *a_out,
                                             double *dt_out)
{
    if (!spec || n_steps < 1 || !a_gauss || !a_in || !a_out || !dt_out || !spec_ok(*spec))
        return DSP_E_INVALID;
    const double dt = spec->T / static_cast<double>(n_steps);
    const double c1 = 0.5 - std::sqrt(3.0) / 6.0, c2 = 0.5 + std::sqrt(3.0) / 6.0;
    for (int64_t n = 0; n < n_steps; ++n) {
        pulse_at(*spec, (static_cast<double>(n) + c1) * dt, a_gauss + 4 * n);
        pulse_at(*spec, (static_cast<double>(n) + c2) * dt, a_gauss + 4 * n + 2);
    }
    pulse_at(*spec, 0.0, a_in);
    pulse_at(*spec, spec->T, a_out);
    *dt_out = dt;
    return DSP_OK;
}

extern "C" dsp_status dsp_sample_pulse(const dsp_pulse_spec *spec, int64_t n_steps,
                                       double *a_mid, double *a_in, double *a_out,
                                       double *dt_out)
{
    if (!spec || n_steps < 1 || !a_mid || !a_in || !a_out || !dt_out || !spec_ok(*spec))
        return DSP_E_INVALID;
    const double dt = spec->T / static_cast<double>(n_steps);
    for (int64_t n = 0; n < n_steps; ++n)
        pulse_at(*spec, (static_cast<double>(n) + 0.5) * dt, a_mid + 2 * n);
    pulse_at(*spec, 0.0, a_in);
    pulse_at(*spec, spec->T, a_out);
    *dt_out = dt;
    return DSP_OK;
}

// ===========================================================================
// Continuous-batching server
//
// Pipelined: dsp_server_step queues iteration k (admissions, one batched
// launch over every admitted request, the finalize of the requests whose last
// steps are in it, and the copies of their results to pinned host memory),
// records an event, and only then waits for iteration k-1's event to retire
// the requests that finished there.  The GPU therefore always has the next
// iteration queued while the host does its bookkeeping.  Which requests finish
// in an iteration is known on the host from the step counts, so no read-back
// is needed to plan the next one.  Device memory comes from the stream-ordered
// pool (cudaMallocAsync / cudaFreeAsync on the server stream), table uploads go
// through pinned staging on a side stream, so no step blocks on an allocation.
// ===========================================================================

namespace {

struct ServerReq {
    int64_t id = 0;
    dsp_request p{};
    std::vector<double> a_mid;
    int32_t state = DSP_REQ_QUEUED;
    dsp_grid g{};             // pointers borrowed from `block`
    void *block = nullptr;    // one pool allocation: state | table | partials | scalars | map
    void *map_dev = nullptr;
    int64_t footprint = 0;
    int64_t finish_iter = -1;  // iteration whose launch holds the last steps
    bool cancel_pending = false;
    int32_t slot = -1;                   // index into the server's pinned result slots
    void *map_host = nullptr;            // pinned, when keep_map
    double density = 0.0;
};

size_t align256(size_t x) { return (x + 255) & ~static_cast<size_t>(255); }

int64_t footprint_of(const dsp_request &p)
{
    const int64_t pts = static_cast<int64_t>(p.nx) * p.ny;
    const int64_t parts = (pts + dsp::kGranule - 1) / dsp::kGranule;
    const size_t nodes = sizeof(float2) * (static_cast<size_t>(p.nx) + static_cast<size_t>(p.ny));
    return static_cast<int64_t>(align256(32 * static_cast<size_t>(pts)) +
                                align256(table_bytes(p.precision, p.scheme, p.n_steps) + nodes) +
                                align256(8 * static_cast<size_t>(parts)) +
                                align256(sizeof(DeviceScalars)) +
                                align256(map_elem_bytes(p.precision) * static_cast<size_t>(pts)));
}

}  // namespace

struct dsp_server {
    int64_t budget = 0, used = 0;
    int32_t max_active = 1;
    int64_t chunk = 1;
    cudaStream_t stream = nullptr;       // compute (caller's)
    cudaStream_t copy_stream = nullptr;  // table uploads
    cudaEvent_t upload_done = nullptr;
    cudaEvent_t iter_done[2] = {nullptr, nullptr};
    int64_t iter = 0;                    // iterations queued so far
    unsigned char *staging = nullptr;    // pinned table staging
    size_t staging_cap = 0;
    int *err = nullptr;                  // device error word of the batched launches
    int *err_host = nullptr;             // pinned copy, refreshed every iteration
    DeviceScalars *slots = nullptr;      // pinned, 2 * max_active: results of two iterations
    std::vector<std::unique_ptr<ServerReq>> reqs;  // by id
    std::deque<int64_t> queue;
    std::vector<int64_t> active;         // admitted, not yet retired
    dsp_status latched = DSP_OK;
};

namespace {

dsp_status server_fail(dsp_server *s, dsp_status st)
{
    cudaGetLastError();
    if (s->latched == DSP_OK)
        s->latched = st;
    return st;
}

void server_release(dsp_server *s, ServerReq *r)
{
    if (r->block) {
        cudaFreeAsync(r->block, s->stream);
        r->block = nullptr;
    }
    r->map_dev = nullptr;
    s->used -= r->footprint;
    r->footprint = 0;
}

// Allocates from the pool and queues the table upload of one request.
dsp_status server_admit(dsp_server *s, ServerReq *r)
{
    const dsp_request &p = r->p;
    fill_grid(&r->g, p.nx, p.ny, p.px_min, p.px_max, p.py_min, p.py_max, p.precision, p.scheme,
              p.valley, s->stream);
    std::vector<unsigned char> host;
    std::vector<float2> nodes;
    dsp_status st =
        prepare_pulse(&r->g, r->a_mid.data(), p.n_steps, p.dt, p.a_in, p.a_out, host, nodes);
    if (st != DSP_OK)
        return st;
    r->g.keep_final_state = false;  // a finished request's state is never read again
    // table (padded to 16 bytes) and projection nodes, uploaded in one copy
    const size_t tb = table_bytes(p.precision, p.scheme, p.n_steps);
    host.resize(tb + node_bytes(&r->g), 0);
    std::memcpy(host.data() + tb, nodes.data(), node_bytes(&r->g));
    const size_t pts = static_cast<size_t>(r->g.n_points);
    const size_t o_table = align256(32 * pts);
    const size_t o_part = o_table + align256(host.size());
    const size_t o_scal = o_part + align256(8 * static_cast<size_t>(r->g.n_parts));
    const size_t o_map = o_scal + align256(sizeof(DeviceScalars));
    const size_t total = o_map + align256(map_elem_bytes(p.precision) * pts);
    // allocated in stream order on the copy stream, so the upload does not wait for
    // the iteration in flight on the compute stream; the compute stream waits for
    // the upload before its first use, and frees the block after its last use
    void *block = nullptr;
    if (cudaMallocAsync(&block, total, s->copy_stream) != cudaSuccess) {
        cudaGetLastError();
        return DSP_E_NOMEM;
    }
    unsigned char *b = static_cast<unsigned char *>(block);
    r->block = block;
    r->g.state = b;
    r->g.table = b + o_table;
    r->g.table_cap = p.n_steps;
    r->g.nodes = reinterpret_cast<float2 *>(b + o_table + tb);
    r->g.partials = reinterpret_cast<double *>(b + o_part);
    r->g.scal = reinterpret_cast<DeviceScalars *>(b + o_scal);
    r->map_dev = b + o_map;
    if (p.keep_map && !r->map_host) {
        if (cudaMallocHost(&r->map_host, map_elem_bytes(p.precision) * pts) != cudaSuccess) {
            cudaGetLastError();
            r->map_host = nullptr;
            cudaFreeAsync(block, s->copy_stream);
            r->block = nullptr;
            return DSP_E_NOMEM;
        }
    }
    // table: host -> pinned staging -> device on the copy stream; the compute
    // stream waits for it before the first launch
    if (!host.empty()) {
        if (cudaEventSynchronize(s->upload_done) != cudaSuccess)  // staging free again
            return server_fail(s, DSP_E_CUDA);
        if (host.size() > s->staging_cap) {
            if (s->staging)
                cudaFreeHost(s->staging);
            s->staging = nullptr;
            s->staging_cap = 0;
            if (cudaMallocHost(reinterpret_cast<void **>(&s->staging), host.size()) != cudaSuccess)
                return server_fail(s, DSP_E_NOMEM);
            s->staging_cap = host.size();
        }
        std::memcpy(s->staging, host.data(), host.size());
        if (cudaMemcpyAsync(r->g.table, s->staging, host.size(), cudaMemcpyHostToDevice,
                            s->copy_stream) != cudaSuccess ||
            cudaEventRecord(s->upload_done, s->copy_stream) != cudaSuccess ||
            cudaStreamWaitEvent(s->stream, s->upload_done, 0) != cudaSuccess)
            return server_fail(s, DSP_E_CUDA);
    }
    if (host.empty() && (cudaEventRecord(s->upload_done, s->copy_stream) != cudaSuccess ||
                         cudaStreamWaitEvent(s->stream, s->upload_done, 0) != cudaSuccess))
        return server_fail(s, DSP_E_CUDA);
    r->footprint = footprint_of(p);
    s->used += r->footprint;
    r->state = DSP_REQ_ACTIVE;
    std::vector<double>().swap(r->a_mid);  // the device holds the table now
    return DSP_OK;
}

}  // namespace

extern "C" {

dsp_status dsp_server_create(int64_t hbm_budget_bytes, int32_t max_active, int64_t chunk_steps,
                             void *cuda_stream, dsp_server **out)
{
    if (!out)
        return DSP_E_INVALID;
    *out = nullptr;
    if (hbm_budget_bytes <= 0 || max_active < 1 || chunk_steps < 1)
        return DSP_E_INVALID;
    dsp_server *s = new (std::nothrow) dsp_server();
    if (!s)
        return DSP_E_NOMEM;
    s->budget = hbm_budget_bytes;
    s->max_active = max_active;
    // whole step groups per launch, so a request meets the same groups alone or in a mix
    s->chunk = chunk_steps >= dsp::kGroupMax
                   ? chunk_steps - chunk_steps % dsp::kGroupMax : chunk_steps;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&s->upload_done, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&s->iter_done[0], cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&s->iter_done[1], cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&s->err), sizeof(int));
    if (e == cudaSuccess)
        e = cudaMallocHost(reinterpret_cast<void **>(&s->err_host), sizeof(int));
    if (e == cudaSuccess)
        e = cudaMallocHost(reinterpret_cast<void **>(&s->slots),
                           sizeof(DeviceScalars) * 2 * static_cast<size_t>(max_active));
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
    if (e == cudaSuccess)
        e = cudaEventRecord(s->upload_done, s->copy_stream);
    if (e == cudaSuccess) {
        // keep freed pool memory in the pool (no return to the driver at syncs)
        int dev = 0;
        cudaMemPool_t pool;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
        cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        dsp_server_destroy(s);
        return DSP_E_CUDA;
    }
    *s->err_host = 0;
    *out = s;
    return DSP_OK;
}

dsp_status dsp_server_submit(dsp_server *s, const dsp_request *req, const double *a_mid,
                             int64_t *id)
{
    if (!s || !req || !id)
        return DSP_E_INVALID;
    if (s->latched != DSP_OK)
        return s->latched;
    const dsp_request &p = *req;
    dsp_status st = validate_grid_args(p.nx, p.ny, p.px_min, p.px_max, p.py_min, p.py_max,
                                       p.precision, p.scheme, p.valley);
    if (st != DSP_OK)
        return st;
    if (p.keep_map != 0 && p.keep_map != 1)
        return DSP_E_INVALID;
    dsp_grid probe;  // only the box matters for the step condition
    probe.px_min = p.px_min;
    probe.px_max = p.px_max;
    probe.py_min = p.py_min;
    probe.py_max = p.py_max;
    const int64_t n_samples = p.n_steps * samples_per_step(p.scheme);
    st = validate_pulse_args(&probe, a_mid, n_samples, p.dt, p.a_in, p.a_out);
    if (st != DSP_OK)
        return st;
    if (footprint_of(p) > s->budget)
        return DSP_E_NOMEM;
    std::unique_ptr<ServerReq> r(new (std::nothrow) ServerReq());
    if (!r)
        return DSP_E_NOMEM;
    r->id = static_cast<int64_t>(s->reqs.size());
    r->p = p;
    try {
        r->a_mid.assign(a_mid, a_mid + 2 * n_samples);
    } catch (...) {
        return DSP_E_NOMEM;
    }
    *id = r->id;
    s->queue.push_back(r->id);
    s->reqs.push_back(std::move(r));
    return DSP_OK;
}

dsp_status dsp_server_step(dsp_server *s, int32_t *n_active, int32_t *n_queued,
                           int32_t *n_finished)
{
    Range range_("dsp_server_step");
    if (!s)
        return DSP_E_INVALID;
    if (s->latched != DSP_OK)
        return s->latched;
    const int64_t k = s->iter;
    int32_t finished = 0;
    // 1. drop cancelled queued requests; cancelled active ones stop being
    //    launched and are released below once their last iteration is done
    {
        std::deque<int64_t> q;
        for (int64_t id : s->queue)
            if (s->reqs[id]->state == DSP_REQ_QUEUED)
                q.push_back(id);
        s->queue.swap(q);
    }
    // 2. admit FIFO while the footprint fits and a slot is free
    {
        Range admit_range_("server admit");
        while (!s->queue.empty() && static_cast<int32_t>(s->active.size()) < s->max_active) {
            ServerReq *r = s->reqs[s->queue.front()].get();
            if (s->used + footprint_of(r->p) > s->budget)
                break;
            s->queue.pop_front();
            dsp_status st = server_admit(s, r);
            if (s->latched != DSP_OK)
                return s->latched;
            if (st != DSP_OK) {
                r->state = DSP_REQ_FAILED;
                std::vector<double>().swap(r->a_mid);
                continue;
            }
            s->active.push_back(r->id);
        }
    }
    // 3. iteration k: one batched launch per precision over the running requests
    bool queued_any = false;
    std::vector<dsp::FinDesc> fins;
    std::vector<ServerReq *> finishing;
    for (int prec = 0; prec < 2; ++prec) {
        std::vector<ReqDesc> descs;
        for (int64_t id : s->active) {
            ServerReq *r = s->reqs[id].get();
            dsp_grid &g = r->g;
            if (r->finish_iter >= 0 || r->state != DSP_REQ_ACTIVE || g.precision != prec)
                continue;
            const int64_t end = std::min(g.n_steps, g.cursor + s->chunk);
            const bool fin = (end == g.n_steps);
            descs.push_back(make_desc(&g, g.cursor, end, fin, r->map_dev));
            descs.back().err = s->err;  // one error word for the server's launches
            g.cursor = end;
            g.fresh = false;
            if (fin) {
                r->finish_iter = k;
                fins.push_back(fin_desc(&g));
                finishing.push_back(r);
            }
        }
        if (descs.empty())
            continue;
        queued_any = true;
        if (launch_requests(descs, prec, s->stream) != cudaSuccess)
            return server_fail(s, DSP_E_CUDA);
    }
    if (launch_finalizes(fins, s->stream) != cudaSuccess)
        return server_fail(s, DSP_E_CUDA);
    // results land in pinned slots [(k & 1) * max_active, ...): read when iteration
    // k is retired, at the latest in step k + 1, before step k + 2 reuses them
    int32_t next_slot = static_cast<int32_t>(k & 1) * s->max_active;
    for (ServerReq *r : finishing) {
        r->slot = next_slot++;
        cudaError_t e = cudaMemcpyAsync(&s->slots[r->slot], r->g.scal, sizeof(DeviceScalars),
                                        cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess && r->p.keep_map)
            e = cudaMemcpyAsync(r->map_host, r->map_dev,
                                static_cast<size_t>(r->g.n_points) * map_elem_bytes(r->p.precision),
                                cudaMemcpyDeviceToHost, s->stream);
        if (e != cudaSuccess)
            return server_fail(s, DSP_E_CUDA);
    }
    if (cudaMemcpyAsync(s->err_host, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaEventRecord(s->iter_done[k & 1], s->stream) != cudaSuccess)
        return server_fail(s, DSP_E_CUDA);
    s->iter = k + 1;
    (void)queued_any;
    // 4. wait for iteration k-1 (k itself when nothing new was queued, so the
    //    loop always makes progress) and retire what finished by then
    const int64_t done_iter = queued_any ? k - 1 : k;
    if (done_iter >= 0) {
        if (cudaEventSynchronize(s->iter_done[done_iter & 1]) != cudaSuccess)
            return server_fail(s, DSP_E_CUDA);
        if (*s->err_host & dsp::kErrTimeout)
            return server_fail(s, DSP_E_TIMEOUT);
        if (*s->err_host & dsp::kErrBounds)
            return server_fail(s, DSP_E_BOUNDS);
        std::vector<int64_t> keep;
        for (int64_t id : s->active) {
            ServerReq *r = s->reqs[id].get();
            const bool launched_out = r->finish_iter >= 0 && r->finish_iter <= done_iter;
            const bool cancelled = r->state == DSP_REQ_CANCELLED;
            if (launched_out || cancelled) {
                if (launched_out && !cancelled) {
                    r->density = s->slots[r->slot].density;
                    r->state = DSP_REQ_DONE;
                }
                server_release(s, r);
                ++finished;
            } else {
                keep.push_back(id);
            }
        }
        s->active.swap(keep);
    }
    if (n_active)
        *n_active = static_cast<int32_t>(s->active.size());
    if (n_queued)
        *n_queued = static_cast<int32_t>(s->queue.size());
    if (n_finished)
        *n_finished = finished;
    return DSP_OK;
}

dsp_status dsp_server_query(dsp_server *s, int64_t id, int32_t *state, double *density,
                            void *map_host, int64_t *steps_done)
{
    if (!s || id < 0 || id >= static_cast<int64_t>(s->reqs.size()) || !state)
        return DSP_E_INVALID;
    ServerReq *r = s->reqs[id].get();
    *state = r->state;
    if (steps_done)
        *steps_done = r->state == DSP_REQ_DONE ? r->p.n_steps : r->g.cursor;
    if (r->state == DSP_REQ_DONE) {
        if (density)
            *density = r->density;
        if (map_host && r->map_host)
            std::memcpy(map_host, r->map_host,
                        static_cast<size_t>(r->p.nx) * r->p.ny * map_elem_bytes(r->p.precision));
    }
    return DSP_OK;
}

dsp_status dsp_server_cancel(dsp_server *s, int64_t id)
{
    if (!s || id < 0 || id >= static_cast<int64_t>(s->reqs.size()))
        return DSP_E_INVALID;
    ServerReq *r = s->reqs[id].get();
    if (r->state == DSP_REQ_QUEUED || r->state == DSP_REQ_ACTIVE) {
        r->state = DSP_REQ_CANCELLED;
        std::vector<double>().swap(r->a_mid);
        return DSP_OK;
    }
    return DSP_E_STATE;
}

dsp_status dsp_server_destroy(dsp_server *s)
{
    if (!s)
        return DSP_OK;
    if (s->latched != DSP_E_CUDA)
        cudaStreamSynchronize(s->stream);
    for (auto &r : s->reqs) {
        if (r->block)
            server_release(s, r.get());
        if (r->map_host)
            cudaFreeHost(r->map_host);
    }
    if (s->latched != DSP_E_CUDA)
        cudaStreamSynchronize(s->stream);
    if (s->copy_stream) {
        cudaStreamSynchronize(s->copy_stream);
        cudaStreamDestroy(s->copy_stream);
    }
    for (cudaEvent_t ev : {s->upload_done, s->iter_done[0], s->iter_done[1]})
        if (ev)
            cudaEventDestroy(ev);
    if (s->staging)
        cudaFreeHost(s->staging);
    if (s->err)
        cudaFree(s->err);
    if (s->err_host)
        cudaFreeHost(s->err_host);
    if (s->slots)
        cudaFreeHost(s->slots);
    delete s;
    return DSP_OK;
}

}  // extern "C"
