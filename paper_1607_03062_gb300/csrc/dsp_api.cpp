// dsp_api.cpp -- host side of the C ABI declared in include/dsp.h: grid
// handles, pulse tables, launches, the density reduction, the pulse sampler and
// the continuous-batching server.
//
// The hot path runs entirely in the kernels of dsp_kernels.cu; this file only
// validates, lays out the per-step table in the layout the kernels read, and
// queues work on the caller's CUDA stream.

#include <cuda_runtime.h>

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

struct DeviceScalars {
    double density;
    int err;
    int pad;
};

}  // namespace

struct dsp_grid {
    int32_t nx = 0, ny = 0, precision = 0, scheme = 0, valley = 1;
    double px_min = 0, px_max = 0, py_min = 0, py_max = 0, hx = 0, hy = 0;
    int64_t n_points = 0;
    int32_t n_tiles = 0;
    cudaStream_t stream = nullptr;

    void *state = nullptr;
    bool owns_state = false;
    void *table = nullptr;
    int64_t table_cap = 0;  // entries
    double *partials = nullptr;
    DeviceScalars *scal = nullptr;
    void *own_map = nullptr;  // used by dsp_solve when the caller passes no map

    bool has_pulse = false;
    int64_t n_steps = 0, cursor = 0;
    double dt = 0, a_in[2] = {0, 0}, a_out[2] = {0, 0};
    double quant = 1, inv_quant = 1;
    int32_t level = 0;
    double theta_max = 0.0;
    bool fresh = true;      // state not yet written on the device
    bool projected = false;  // partial sums valid for the current pulse
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
// ~theta ds_err.  The budget over n_steps steps is 2e-8 (FP32_MIXED, well below
// its 1e-5 target) or 1e-16 (FP64).
int32_t choose_level(int32_t precision, double theta, int64_t n_steps)
{
    const double x = theta * theta;
    const double budget =
        (precision == DSP_FP64 ? 1e-16 : 2e-8) / static_cast<double>(std::max<int64_t>(n_steps, 1));
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

double box_abs_max(const dsp_grid *g)
{
    return std::max(std::max(std::fabs(g->px_min), std::fabs(g->px_max)),
                    std::max(std::fabs(g->py_min), std::fabs(g->py_max)));
}

// dt * max over steps and box corners of |p + A_n| (|P| is convex in p, so the
// maximum over the box is at a corner).
double theta_max(const dsp_grid *g, const double *a_mid, int64_t n, double dt)
{
    double m = 0.0;
    const double cx[2] = {g->px_min, g->px_max}, cy[2] = {g->py_min, g->py_max};
    for (int64_t k = 0; k < n; ++k)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j)
                m = std::max(m, std::hypot(cx[i] + a_mid[2 * k], cy[j] + a_mid[2 * k + 1]));
    return dt * m;
}

// 2^k such that hi parts (multiples of 2^-k) of dt*p and dt*A, and their sum,
// are exact in FP32: |hi| <= B and |sum| < 2B + 2^-k < 2^(24-k).
double choose_quant(const dsp_grid *g, const double *a_mid, int64_t n, double dt)
{
    double b = box_abs_max(g);
    for (int64_t k = 0; k < 2 * n; ++k)
        b = std::max(b, std::fabs(a_mid[k]));
    b *= dt;
    if (!(b > 0.0))
        return 1.0;
    int e = 0;
    (void)std::frexp(2.0 * b, &e);  // 2b < 2^e
    return std::ldexp(1.0, 23 - e);
}

dsp_status check_usable(const dsp_grid *g)
{
    if (!g)
        return DSP_E_INVALID;
    return g->latched;
}

ReqDesc make_desc(const dsp_grid *g, int64_t begin, int64_t end, bool project, void *map)
{
    ReqDesc r;
    std::memset(&r, 0, sizeof(r));
    r.table = g->table;
    r.state = g->state;
    r.map = map;
    r.partials = g->partials;
    r.px_min = g->px_min;
    r.py_min = g->py_min;
    r.hx = g->hx;
    r.hy = g->hy;
    r.dt = g->dt;
    r.a_in[0] = g->a_in[0];
    r.a_in[1] = g->a_in[1];
    r.a_out[0] = g->a_out[0];
    r.a_out[1] = g->a_out[1];
    r.quant = g->quant;
    r.inv_quant = g->inv_quant;
    r.n_points = g->n_points;
    r.step_begin = begin;
    r.step_end = end;
    r.nx = g->nx;
    r.ny = g->ny;
    r.scheme = g->scheme;
    r.valley = g->valley;
    r.level = g->level;
    r.fresh = g->fresh ? 1 : 0;
    r.project = project ? 1 : 0;
    r.n_tiles = g->n_tiles;
    return r;
}

double density_scale(const dsp_grid *g)
{
    return 4.0 / ((2.0 * kPi) * (2.0 * kPi)) * g->hx * g->hy;
}

// Queues launches advancing several requests of one precision; requests are
// split into launches of at most kMaxReqPerLaunch.
cudaError_t launch_requests(const std::vector<ReqDesc> &reqs, int precision, int *err,
                            cudaStream_t stream)
{
    size_t i = 0;
    while (i < reqs.size()) {
        std::unique_ptr<EvolveArgs> a(new EvolveArgs());
        std::memset(a.get(), 0, sizeof(EvolveArgs));
        a->err = err;
        int tiles = 0;
        int n = 0;
        while (i < reqs.size() && n < dsp::kMaxReqPerLaunch) {
            a->r[n] = reqs[i];
            a->r[n].tile_begin = tiles;
            tiles += reqs[i].n_tiles;
            ++n;
            ++i;
        }
        a->nreq = n;
        a->total_tiles = tiles;
        cudaError_t e = dsp::launch_evolve(*a, precision, stream);
        if (e != cudaSuccess)
            return e;
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
    f.n_tiles = g->n_tiles;
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
    if (scheme != DSP_SCHEME_EXACT && scheme != DSP_SCHEME_STRANG_XY)
        return DSP_E_INVALID;
    if (valley != 1 && valley != -1)
        return DSP_E_INVALID;
    return DSP_OK;
}

dsp_status validate_pulse_args(const dsp_grid *g, const double *a_mid, int64_t n_steps, double dt,
                               const double a_in[2], const double a_out[2])
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
    if (n_steps > 0 && theta_max(g, a_mid, n_steps, dt) > kPi)
        return DSP_E_CFL;
    return DSP_OK;
}

// Fills the table layout the kernels read (see ReqDesc::table).
void build_table(const dsp_grid *g, const double *a_mid, int64_t n, double dt, double quant,
                 double inv_quant, std::vector<unsigned char> &out)
{
    out.resize(static_cast<size_t>(n) * 16);
    // valley K- is stepped as K+ on -P, so its table holds -dt*A
    const double vs = g->valley > 0 ? 1.0 : -1.0;
    if (g->precision == DSP_FP64) {
        double *t = reinterpret_cast<double *>(out.data());
        for (int64_t k = 0; k < n; ++k) {
            t[2 * k] = vs * (dt * a_mid[2 * k]);
            t[2 * k + 1] = vs * (dt * a_mid[2 * k + 1]);
        }
    } else {
        float *t = reinterpret_cast<float *>(out.data());
        for (int64_t k = 0; k < n; ++k) {
            for (int c = 0; c < 2; ++c) {
                const double v = vs * (dt * a_mid[2 * k + c]);
                const double hi = std::rint(v * quant) * inv_quant;
                t[4 * k + 2 * c] = static_cast<float>(hi);
                t[4 * k + 2 * c + 1] = static_cast<float>(v - hi);
            }
        }
    }
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
    g->state = g->table = g->own_map = nullptr;
    g->partials = nullptr;
    g->scal = nullptr;
}

dsp_status create_grid_impl(int32_t nx, int32_t ny, double px_min, double px_max, double py_min,
                            double py_max, int32_t precision, int32_t scheme, int32_t valley,
                            cudaStream_t stream, void *state_dev, int64_t state_bytes,
                            dsp_grid **out)
{
    if (!out)
        return DSP_E_INVALID;
    *out = nullptr;
    dsp_status s =
        validate_grid_args(nx, ny, px_min, px_max, py_min, py_max, precision, scheme, valley);
    if (s != DSP_OK)
        return s;
    const int64_t need = dsp_state_bytes(nx, ny, precision);
    if (state_dev && (state_bytes < need || (reinterpret_cast<uintptr_t>(state_dev) & 15u)))
        return DSP_E_INVALID;
    dsp_grid *g = new (std::nothrow) dsp_grid();
    if (!g)
        return DSP_E_NOMEM;
    g->nx = nx;
    g->ny = ny;
    g->precision = precision;
    g->scheme = scheme;
    g->valley = valley;
    g->px_min = px_min;
    g->px_max = px_max;
    g->py_min = py_min;
    g->py_max = py_max;
    g->hx = (px_max - px_min) / nx;
    g->hy = (py_max - py_min) / ny;
    g->n_points = static_cast<int64_t>(nx) * ny;
    g->n_tiles = static_cast<int32_t>((g->n_points + dsp::kTilePoints - 1) / dsp::kTilePoints);
    g->stream = stream;
    cudaError_t e = cudaSuccess;
    if (state_dev) {
        g->state = state_dev;
    } else {
        e = cudaMalloc(&g->state, static_cast<size_t>(need));
        g->owns_state = (e == cudaSuccess);
    }
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&g->partials), sizeof(double) * g->n_tiles);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&g->scal), sizeof(DeviceScalars));
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

dsp_status set_pulse_impl(dsp_grid *g, const double *a_mid, int64_t n_steps, double dt,
                          const double a_in[2], const double a_out[2])
{
    dsp_status s = validate_pulse_args(g, a_mid, n_steps, dt, a_in, a_out);
    if (s != DSP_OK)
        return s;
    const double tmax = n_steps > 0 ? theta_max(g, a_mid, n_steps, dt) : 0.0;
    const double quant = n_steps > 0 ? choose_quant(g, a_mid, n_steps, dt) : 1.0;
    std::vector<unsigned char> host;
    build_table(g, a_mid, n_steps, dt, quant, 1.0 / quant, host);
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
            e = cudaMalloc(&g->table, static_cast<size_t>(n_steps) * 16);
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
    g->has_pulse = true;
    g->n_steps = n_steps;
    g->cursor = 0;
    g->dt = dt;
    g->a_in[0] = a_in[0];
    g->a_in[1] = a_in[1];
    g->a_out[0] = a_out[0];
    g->a_out[1] = a_out[1];
    g->quant = quant;
    g->inv_quant = 1.0 / quant;
    g->theta_max = tmax;
    g->level = choose_level(g->precision, tmax, n_steps);
    g->fresh = true;
    g->projected = false;
    return DSP_OK;
}

// Advances one grid to `end`, optionally projecting into `map` at the end.
dsp_status run_one(dsp_grid *g, int64_t end, bool project, void *map)
{
    std::vector<ReqDesc> r(1, make_desc(g, g->cursor, end, project, map));
    cudaError_t e = launch_requests(r, g->precision, &g->scal->err, g->stream);
    if (e != cudaSuccess)
        return latch_cuda(g, e);
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

dsp_status dsp_set_pulse(dsp_grid *g, const double *a_mid, int64_t n_steps, double dt,
                         const double a_in[2], const double a_out[2])
{
    dsp_status s = check_usable(g);
    if (s != DSP_OK)
        return s;
    return set_pulse_impl(g, a_mid, n_steps, dt, a_in, a_out);
}

dsp_status dsp_evolve(dsp_grid *g, int64_t steps)
{
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
        cudaError_t e = launch_requests(reqs, prec, &grids[0]->scal->err, grids[0]->stream);
        if (e != cudaSuccess) {
            for (int32_t i = 0; i < count; ++i)
                latch_cuda(grids[i], e);
            return DSP_E_CUDA;
        }
    }
    for (int32_t i = 0; i < count; ++i) {
        if (steps[i] == 0)
            continue;
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
    info->n_tiles = g->n_tiles;
    info->dt = g->dt;
    info->theta_max = g->theta_max;
    info->quant = g->quant;
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
    if (!g->has_pulse)
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
// ===========================================================================

namespace {

struct ServerReq {
    int64_t id = 0;
    dsp_request p{};
    std::vector<double> a_mid;
    int32_t state = DSP_REQ_QUEUED;
    dsp_grid *g = nullptr;
    void *map_dev = nullptr;
    int64_t footprint = 0;
    std::vector<unsigned char> map_host;
    double density = 0.0;
    bool finishing = false;
};

int64_t footprint_of(const dsp_request &p)
{
    const int64_t pts = static_cast<int64_t>(p.nx) * p.ny;
    const int64_t tiles = (pts + dsp::kTilePoints - 1) / dsp::kTilePoints;
    return 32 * pts + 16 * p.n_steps + static_cast<int64_t>(map_elem_bytes(p.precision)) * pts +
           8 * tiles + static_cast<int64_t>(sizeof(DeviceScalars));
}

}  // namespace

struct dsp_server {
    int64_t budget = 0, used = 0;
    int32_t max_active = 1;
    int64_t chunk = 1;
    cudaStream_t stream = nullptr;
    std::vector<std::unique_ptr<ServerReq>> reqs;  // by id
    std::deque<int64_t> queue;
    std::vector<int64_t> active;
    int *err = nullptr;  // device error word of the batched launches
    dsp_status latched = DSP_OK;
};

namespace {

void server_release(dsp_server *s, ServerReq *r)
{
    if (r->g) {
        dsp_destroy_grid(r->g);
        r->g = nullptr;
    }
    if (r->map_dev) {
        cudaFree(r->map_dev);
        r->map_dev = nullptr;
    }
    s->used -= r->footprint;
    r->footprint = 0;
}

// Allocates and uploads one request; false if the device refused memory.
dsp_status server_admit(dsp_server *s, ServerReq *r)
{
    const dsp_request &p = r->p;
    dsp_status st = create_grid_impl(p.nx, p.ny, p.px_min, p.px_max, p.py_min, p.py_max,
                                     p.precision, p.scheme, p.valley, s->stream, nullptr, 0, &r->g);
    if (st != DSP_OK)
        return st;
    const size_t mb = static_cast<size_t>(r->g->n_points) * map_elem_bytes(p.precision);
    if (cudaMalloc(&r->map_dev, mb) != cudaSuccess) {
        cudaGetLastError();
        r->map_dev = nullptr;
        dsp_destroy_grid(r->g);
        r->g = nullptr;
        return DSP_E_NOMEM;
    }
    st = set_pulse_impl(r->g, r->a_mid.data(), p.n_steps, p.dt, p.a_in, p.a_out);
    if (st != DSP_OK) {
        cudaFree(r->map_dev);
        r->map_dev = nullptr;
        dsp_destroy_grid(r->g);
        r->g = nullptr;
        return st;
    }
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
    s->chunk = chunk_steps;
    s->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&s->err), sizeof(int));
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->err, 0, sizeof(int), s->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (s->err)
            cudaFree(s->err);
        delete s;
        return DSP_E_NOMEM;
    }
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
    st = validate_pulse_args(&probe, a_mid, p.n_steps, p.dt, p.a_in, p.a_out);
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
        r->a_mid.assign(a_mid, a_mid + 2 * p.n_steps);
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
    if (!s)
        return DSP_E_INVALID;
    if (s->latched != DSP_OK)
        return s->latched;
    int32_t finished = 0;
    // 1. drop cancelled requests
    {
        std::vector<int64_t> keep;
        for (int64_t id : s->active) {
            ServerReq *r = s->reqs[id].get();
            if (r->state == DSP_REQ_CANCELLED)
                server_release(s, r);
            else
                keep.push_back(id);
        }
        s->active.swap(keep);
        std::deque<int64_t> q;
        for (int64_t id : s->queue)
            if (s->reqs[id]->state == DSP_REQ_QUEUED)
                q.push_back(id);
        s->queue.swap(q);
    }
    // 2. admit FIFO while the footprint fits and a slot is free
    while (!s->queue.empty() && static_cast<int32_t>(s->active.size()) < s->max_active) {
        ServerReq *r = s->reqs[s->queue.front()].get();
        if (s->used + footprint_of(r->p) > s->budget)
            break;
        s->queue.pop_front();
        dsp_status st = server_admit(s, r);
        if (st != DSP_OK) {
            r->state = DSP_REQ_FAILED;
            continue;
        }
        s->active.push_back(r->id);
    }
    // 3. one batched launch per precision over every active request
    if (!s->active.empty()) {
        std::vector<dsp::FinDesc> fins;
        for (int prec = 0; prec < 2; ++prec) {
            std::vector<ReqDesc> descs;
            for (int64_t id : s->active) {
                ServerReq *r = s->reqs[id].get();
                dsp_grid *g = r->g;
                if (g->precision != prec)
                    continue;
                const int64_t end = std::min(g->n_steps, g->cursor + s->chunk);
                r->finishing = (end == g->n_steps);
                descs.push_back(make_desc(g, g->cursor, end, r->finishing, r->map_dev));
                if (r->finishing)
                    fins.push_back(fin_desc(g));
            }
            if (descs.empty())
                continue;
            cudaError_t e = launch_requests(descs, prec, s->err, s->stream);
            if (e != cudaSuccess) {
                s->latched = DSP_E_CUDA;
                return DSP_E_CUDA;
            }
        }
        cudaError_t e = launch_finalizes(fins, s->stream);
        // 4. copy results of the finishing requests back
        std::vector<DeviceScalars> hs(s->active.size());
        size_t k = 0;
        for (int64_t id : s->active) {
            ServerReq *r = s->reqs[id].get();
            dsp_grid *g = r->g;
            const int64_t end = std::min(g->n_steps, g->cursor + s->chunk);
            g->cursor = end;
            g->fresh = false;
            if (!r->finishing || e != cudaSuccess) {
                ++k;
                continue;
            }
            g->projected = true;
            e = cudaMemcpyAsync(&hs[k], g->scal, sizeof(DeviceScalars), cudaMemcpyDeviceToHost,
                                s->stream);
            if (e == cudaSuccess && r->p.keep_map) {
                const size_t mb = static_cast<size_t>(g->n_points) * map_elem_bytes(g->precision);
                try {
                    r->map_host.resize(mb);
                } catch (...) {
                    r->state = DSP_REQ_FAILED;
                }
                if (r->state != DSP_REQ_FAILED)
                    e = cudaMemcpyAsync(r->map_host.data(), r->map_dev, mb, cudaMemcpyDeviceToHost,
                                        s->stream);
            }
            ++k;
        }
        int herr = 0;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&herr, s->err, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) {
            s->latched = DSP_E_CUDA;
            return DSP_E_CUDA;
        }
        if (herr & dsp::kErrTimeout) {
            s->latched = DSP_E_TIMEOUT;
            return DSP_E_TIMEOUT;
        }
        // 5. retire
        std::vector<int64_t> keep;
        k = 0;
        for (int64_t id : s->active) {
            ServerReq *r = s->reqs[id].get();
            if (r->finishing) {
                if (hs[k].err & dsp::kErrTimeout) {
                    r->state = DSP_REQ_FAILED;
                } else if (r->state != DSP_REQ_FAILED) {
                    r->density = hs[k].density;
                    r->state = DSP_REQ_DONE;
                }
                server_release(s, r);
                ++finished;
            } else {
                keep.push_back(id);
            }
            ++k;
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
        *steps_done = r->state == DSP_REQ_DONE ? r->p.n_steps : (r->g ? r->g->cursor : 0);
    if (r->state == DSP_REQ_DONE) {
        if (density)
            *density = r->density;
        if (map_host && !r->map_host.empty())
            std::memcpy(map_host, r->map_host.data(), r->map_host.size());
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
    for (auto &r : s->reqs)
        if (r->g || r->map_dev)
            server_release(s, r.get());
    if (s->err)
        cudaFree(s->err);
    delete s;
    return DSP_OK;
}

}  // extern "C"
