// lpm_api.cu - the C ABI (include/lpm.h): context, inputs, stepping, read-backs.
//
// Host-side bookkeeping only: validation, device allocations, the release tables
// (initial mass per release step, fixed-point scale) and the segmentation of a run at
// the binning steps. Every arithmetic step of the particle method runs in the kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>
#include <algorithm>

#include "../../include/lpm.h"
#include "lpm_launch.h"
#include "lpm_adjoint.h"

using namespace lpm;

namespace {

thread_local std::string g_create_error;

struct ScenHost {
    bool released = false;
    double src_x = 0, src_y = 0, src_z = 0;
    long long first_slot = 0;        // state slot of the held range's first particle
    long long n = 0;                 // particles held by this context
    long long n_total = 0;           // particles of the whole release
    long long part_first = 0;        // index of the held range's first particle
    long long id_base = 0;           // global id of the release's particle 0
    long long rel_first = 0, rel_last = 0;
    std::vector<double> q;
    double q_dt = 3600.0;
    int shift = 0;
    double total_mass = 0.0;
    std::vector<double> m0;          // per release step (FP64, host)
    std::vector<float> wind_offset;  // [n_met_t][2] or empty
    double mode_phase[MAX_MODES] = {};   // this scenario's realisation of the perturbation
    double mode_amp[MAX_MODES] = {};     // modes (cycles, m/s); amplitude 0 = mode off
};

}  // namespace

struct lpm_ctx {
    lpm_config cfg{};
    std::vector<double> zlev;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;      // private stream the batched graphs are captured on
    int device = 0;
    int sm_count = 0;
    std::string err;

    // weather
    float4 *d_uvwk = nullptr;               // slabs as given [n_t][nodes]
    float *d_kh = nullptr;
    float4 *d_pair = nullptr;               // time-paired slabs [n_pair][nodes][2]
    float2 *d_khpair = nullptr;             // [n_pair][nodes]
    uint8_t *d_rain = nullptr;
    std::vector<char> met_set;
    bool any_rain = false;
    // asynchronous weather uploads from page-locked host memory
    cudaStream_t copy_stream = nullptr;
    // the adjoint's checkpoint form recomputes the next segment on its own stream while the
    // current one is swept; events: a scratch half recomputed (ev_adj[0..1]) and swept
    // (ev_adj[2..3]), and the sweep's start (ev_adj[4])
    cudaStream_t adj_stream = nullptr;
    cudaEvent_t ev_adj[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_main = nullptr;          // orders a copy after the context stream's work
    std::vector<cudaEvent_t> ev_pair;       // time pair h packed (copy stream)
    std::vector<char> pair_pending;
    // boundary-layer columns for K_z from Eq. 3
    int kz_model = 0;                       // 0: gridded K_z, 1: Eq. 3
    double kz_min = 0.1;
    float4 *d_bl = nullptr;                 // [n_t][ny][nx] (u*, 1/L, H_z, 0) as given
    float4 *d_blpair = nullptr;             // [n_pair][ny][nx][2] value + difference
    std::vector<char> bl_set;

    // particles and outputs
    float4 *d_state = nullptr;
    unsigned long long *d_conc = nullptr;   // [n_scen][cz*cy*cx]
    unsigned long long *d_dep = nullptr;    // [n_scen][2*cy*cx]
    unsigned long long *d_ctr = nullptr;    // [N_COUNTERS][n_scen]
    unsigned int *d_err = nullptr;
    unsigned int *d_queue = nullptr;
    float *d_m0 = nullptr;
    size_t d_m0_cap = 0;
    unsigned char *d_zlut = nullptr;        // vertical level lookup table
    int n_lut = 0;
    float lut_z0 = 0.f, lut_inv_h = 0.f;
    ScenDev *d_scen = nullptr;
    float2 *d_woff = nullptr;               // [n_scen][n_met_t]
    bool any_woff = false;                  // some scenario has a wind offset
    Tile *d_tiles = nullptr;
    size_t d_tiles_cap = 0;

    std::vector<ScenHost> scen;
    int n_released = 0;
    long long n_slots_used = 0;
    long long n_ids_used = 0;               // next global id for lpm_release
    bool profiling = false;
    long long n_launches = 0;               // kernels launched by this context
    long long n_adv_launches = 0;
    double adv_ms = 0.0;                    // device time of advance launches (profiling)
    std::vector<cudaEvent_t> ev_pool;       // profiling events, reused
    size_t ev_used = 0;
    bool tables_dirty = true;
    long long k = 0;                        // steps taken
    long long n_bins = 0;                   // snapshots taken
    int block = 512, ppt = 1, occ = 2;

    // sorting by weather cell (both forms) at the multiples of sort_every: d_state is the
    // home buffer (slot order of the API); the live particles released before sorted_upto
    // sit ordered by cell in d_sorted[cur], the dead ones in d_grave
    int sort_every = 60;                    // steps between sorts; 0 = off
    long long sorted_upto = 0;
    int cur = 0;
    float4 *d_sorted[2] = {nullptr, nullptr};
    unsigned int *d_pidx[2] = {nullptr, nullptr};   // home slot of each sorted slot
    unsigned int *d_slot_of = nullptr;      // per home slot: sorted slot, grave index or home
    unsigned int *d_keys = nullptr;
    size_t keys_cap = 0;
    unsigned int *d_hist = nullptr, *d_bsums = nullptr, *d_live = nullptr;   // d_live = meta[4]
    float4 *d_grave = nullptr;              // particles found dead at a sort (read-back only)
    unsigned int *d_grave_n = nullptr;
    unsigned int *d_grave_home = nullptr;   // home slot of each entry of d_grave
    bool slot_map_stale = false;            // d_slot_of predates the last sort

    // decay chain (species 1..: daughters)
    int n_species = 1;
    double chain_c[MAX_SPECIES][MAX_SPECIES] = {};
    double chain_l[MAX_SPECIES] = {};
    unsigned long long *d_sp_conc = nullptr;  // [n_species-1][n_scen][cz*cy*cx]
    unsigned long long *d_sp_dep = nullptr;   // [n_species-1][n_scen][2*cy*cx]

    // vertical Langevin variant: turbulent velocity per particle (home and sorted slots)
    int langevin = 0;
    double t_lagr = 100.0;
    float *d_w_home = nullptr;
    float *d_w_sorted[2] = {nullptr, nullptr};

    // perturbation modes of the scenarios' wind: shared waves and height profile, the
    // scenarios' phases and amplitudes on the device as 32-byte rows
    int n_modes = 0;
    double modes[MAX_MODES][5] = {};        // (fx, fy, omega, eu, ev)
    std::vector<double> mode_profile;       // [nz]
    float *d_mode_sc = nullptr;             // [n_scen][8]

    // time-integrated dosage
    unsigned long long *d_dose = nullptr;   // [n_scen][cz*cy*cx]
    int dose_every = 0;
    int dose_bits = 0;                      // ceil(log2(floor(n_steps / dose_every)))
    long long n_dose = 0;                   // samples taken since the last (re)start

    // differentiable parameters (adjoint form): diffusivity scale and wind bias
    double k_scale = 1.0, bias_u = 0.0, bias_v = 0.0;
    // receptor / adjoint state
    float *d_mq = nullptr;                  // dt / n_s per release step
    short *d_qi = nullptr;                  // emission-series index per release step
    float4 *d_ckpt = nullptr;
    size_t d_ckpt_cap = 0;
    double *d_conv = nullptr;               // read-back of a grid converted on the device
    size_t d_conv_cap = 0;
    // trajectory storage (the default when it fits): rows of every tile from its first
    // release step on, and the state after each particle's last step (float4 elements)
    float4 *d_traj = nullptr, *d_fin = nullptr;
    size_t d_traj_cap = 0, d_fin_cap = 0;
    longlong2 *d_traj_tile = nullptr;
    size_t traj_need = 0;
    size_t adj_store_max = (size_t)128 << 30;   // bytes; 0 keeps checkpoints only
    bool adj_traj = false;                      // storage of the held forward
    // sorted form (sorting on): CK-step segments over the particles in weather-cell order
    // (several scenarios: scenario, then cell tile), with the adjoint's own sort buffers (the
    // run's sort state is not touched)
    struct AdjSorted {
        std::vector<Tile> tiles;                // release tiles grouped by segment
        std::vector<int> seg_tile;              // [n_seg + 1] first release tile of a segment
        std::vector<int> tiles_a;               // [n_seg] blocks over its sorted entries
        std::vector<long long> off, foff;       // [n_seg + 1] trajectory / end-state offsets
        std::vector<long long> ckoff;           // [n_seg + 1] checkpoint offsets (sorted entries)
        long long max_width = 0;
        Tile *d_tiles = nullptr;
        unsigned int *ord = nullptr, *live = nullptr, *keys = nullptr, *hist = nullptr,
                     *bsums = nullptr, *meta = nullptr, *slot_of = nullptr, *grave_n = nullptr;
        float4 *st[2] = {nullptr, nullptr};
        float4 *home = nullptr, *mu = nullptr, *grave = nullptr;
    } as;
    bool adj_sorted = false;                    // the held forward used the sorted form
                                                // (with adj_traj false: its checkpoint form,
                                                // d_traj / d_fin two segments' scratch)
    float4 *d_rec = nullptr;
    int *d_rbin_off = nullptr;              // receptor bins (AdjParams)
    unsigned char *d_rbin_idx = nullptr;
    size_t d_rbin_off_cap = 0, d_rbin_idx_cap = 0;
    double *d_rC = nullptr, *d_rw = nullptr, *d_rgrad = nullptr;
    size_t d_rbuf_cap = 0;
    Tile *d_adj_tiles = nullptr;
    std::vector<Tile> adj_tiles;
    bool adj_tiles_valid = false;
    std::vector<double> adj_sig;            // signature of the forward whose states are held
    long long params_version = 0;

    // batched form: one CUDA graph per lpm_step call (sorts, memsets, persistent launches),
    // keyed by the steps and the sort state it starts from
    struct Graph {
        long long k0, k1, upto0;
        int cur0;
        long long upto1;
        int cur1;
        long long kernels;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;

    // tile table: runs of at most block*ppt particles of one scenario, grouped by the sort
    // interval [j*E, (j+1)*E) their particles leave in (one interval when sorting is off),
    // ordered by the release step of their first particle within an interval
    std::vector<Tile> tiles;
    std::vector<long long> tile_sp;         // release step of each tile's first particle
    std::vector<int> int_lo;                // first tile of each interval (+ the end)
    long long tiles_E = 1;                  // interval length of the table
    bool tiles_valid = false;

    size_t ncell() const { return (size_t)cfg.cx * cfg.cy * cfg.cz; }
    size_t ndep() const { return (size_t)2 * cfg.cx * cfg.cy; }
};

namespace {

void drop_graphs(lpm_ctx *c);
lpm_status fail(lpm_ctx *c, lpm_status s, const char *fmt, ...) __attribute__((format(printf, 3, 4)));

lpm_status fail(lpm_ctx *c, lpm_status s, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return s;
}

// On failure the CUDA error is reported through the status and consumed, so that it
// does not resurface at a later, unrelated launch check.
#define LPM_CUDA(c, call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (void)cudaGetLastError();                                                      \
            return fail((c), e_ == cudaErrorMemoryAllocation ? LPM_E_OOM : LPM_E_CUDA,     \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                   \
        }                                                                                  \
    } while (0)

bool is_finite(double v) { return std::isfinite(v); }

lpm_status validate(const lpm_config *c)
{
    if (!c) return fail(nullptr, LPM_E_INVALID, "config is NULL");
    if (c->nx < 2 || c->ny < 2 || c->nz < 2)
        return fail(nullptr, LPM_E_INVALID, "met grid needs at least 2 nodes per axis");
    if (c->nz > MAX_LEVELS)
        return fail(nullptr, LPM_E_INVALID, "nz=%d exceeds %d levels", c->nz, MAX_LEVELS);
    if ((double)c->nx * c->ny * c->nz > 1073741824.0)
        return fail(nullptr, LPM_E_INVALID, "met grid exceeds 2^30 nodes");
    if (sort_key_range(c->nx, c->ny, c->nz) >= 0xffffffffLL)
        return fail(nullptr, LPM_E_INVALID, "met grid too large for 32-bit sort keys");
    if (!c->z_levels) return fail(nullptr, LPM_E_INVALID, "z_levels is NULL");
    for (int k = 0; k < c->nz; ++k) {
        if (!is_finite(c->z_levels[k])) return fail(nullptr, LPM_E_INVALID, "z_levels not finite");
        if (k && !(c->z_levels[k] > c->z_levels[k - 1]))
            return fail(nullptr, LPM_E_INVALID, "z_levels must be strictly ascending");
    }
    if (!(c->dx > 0) || !(c->dy > 0) || !is_finite(c->x0) || !is_finite(c->y0))
        return fail(nullptr, LPM_E_INVALID, "met spacing must be > 0");
    if (c->n_met_t < 1 || !(c->met_dt > 0) || !is_finite(c->met_t0))
        return fail(nullptr, LPM_E_INVALID, "need n_met_t >= 1 and met_dt > 0");
    if (c->cx < 1 || c->cy < 1 || c->cz < 1 || !(c->cdx > 0) || !(c->cdy > 0) || !(c->cdz > 0))
        return fail(nullptr, LPM_E_INVALID, "concentration grid must be non-empty");
    if ((double)c->cx * c->cy * c->cz > 2147483647.0)
        return fail(nullptr, LPM_E_INVALID, "concentration grid exceeds 2^31 cells");
    if (!(c->dt > 0) || !is_finite(c->dt)) return fail(nullptr, LPM_E_INVALID, "dt must be > 0");
    if (c->n_steps < 1 || c->n_steps > (int64_t)TAG_STEP)
        return fail(nullptr, LPM_E_INVALID, "n_steps must be in [1, 2^28)");
    if (c->bin_every < 1) return fail(nullptr, LPM_E_INVALID, "bin_every must be >= 1");
    if (c->vd_dry < 0 || c->wet_lambda < 0 || !is_finite(c->vd_dry) || !is_finite(c->wet_lambda))
        return fail(nullptr, LPM_E_INVALID, "deposition parameters must be >= 0");
    if (c->vd_dry > 0 && !(c->h_mix > 0))
        return fail(nullptr, LPM_E_INVALID, "dry deposition needs h_mix > 0");
    if (c->reflect_top && !(c->z_top > 0))
        return fail(nullptr, LPM_E_INVALID, "top reflection needs z_top > 0");
    if (c->n_scenarios < 1) return fail(nullptr, LPM_E_INVALID, "n_scenarios must be >= 1");
    if (c->max_particles < 1 || c->max_particles > 0x7ffffffeLL)
        return fail(nullptr, LPM_E_INVALID, "max_particles must be in [1, 2^31 - 2]");
    return LPM_OK;
}

// Probability of an event per step as a 32-bit threshold (event iff word < T).
unsigned int threshold(double p)
{
    if (!(p > 0.0)) return 0u;
    const double t = std::floor(p * 4294967296.0);
    if (t >= 4294967295.0) return 4294967295u;
    return (unsigned int)t;
}

float pow2f(int e) { return std::ldexp(1.0f, e); }

void fill_params(const lpm_ctx *c, StepParams &P)
{
    const lpm_config &g = c->cfg;
    std::memset(&P, 0, sizeof P);
    P.pair = c->d_pair;
    P.khpair = c->d_khpair;
    P.rain = c->any_rain ? c->d_rain : nullptr;
    P.nx = g.nx; P.ny = g.ny; P.nz = g.nz; P.n_t = g.n_met_t;
    P.slab = (long long)g.nx * g.ny * g.nz;
    P.x0 = (float)g.x0; P.y0 = (float)g.y0;
    P.dx = (float)g.dx; P.dy = (float)g.dy;
    P.inv_dx = (float)(1.0 / g.dx); P.inv_dy = (float)(1.0 / g.dy);
    P.met_t0 = (float)g.met_t0; P.met_dt = (float)g.met_dt;
    P.inv_met_dt = (float)(1.0 / g.met_dt);
    P.x_lo = (float)g.x0; P.x_hi = (float)(g.x0 + (g.nx - 1) * g.dx);
    P.y_lo = (float)g.y0; P.y_hi = (float)(g.y0 + (g.ny - 1) * g.dy);
    for (int k = 0; k < g.nz; ++k) {      // same FP32 arithmetic as a kernel would do
        const float z0 = (float)c->zlev[k];
        const float inv = k + 1 < g.nz ? 1.0f / ((float)c->zlev[k + 1] - z0) : 0.0f;
        P.zi[k] = make_float2(z0, inv);
    }
    P.dt = (float)g.dt;
    P.kh_uniform = (float)g.kh_uniform;
    P.k_scale = (float)c->k_scale;
    P.bias_u = (float)c->bias_u;
    P.bias_v = (float)c->bias_v;
    P.lambda = g.half_life_s > 0 ? (float)(std::log(2.0) / g.half_life_s) : 0.0f;
    P.h_mix = (float)g.h_mix;
    P.z_top = (float)g.z_top;
    P.seed_lo = (unsigned int)(g.seed & 0xffffffffu);
    P.seed_hi = (unsigned int)(g.seed >> 32);
    for (int r = 0; r < 10; ++r) {                  // Philox key schedule (Weyl increments)
        P.rk[2 * r] = P.seed_lo + (unsigned int)r * 0x9E3779B9u;
        P.rk[2 * r + 1] = P.seed_hi + (unsigned int)r * 0xBB67AE85u;
    }
    const double p_dry = (g.vd_dry > 0 && g.h_mix > 0) ? 1.0 - std::exp(-g.vd_dry * g.dt / g.h_mix) : 0.0;
    const double p_wet = (g.wet_lambda > 0 && c->any_rain) ? 1.0 - std::exp(-g.wet_lambda * g.dt) : 0.0;
    P.t_dry = threshold(p_dry);
    P.t_wet = threshold(p_wet);
    P.reflect_ground = g.reflect_ground;
    P.reflect_top = g.reflect_top;
    P.lateral_exit = g.lateral_exit;
    P.drift = g.drift_correction;
    P.cx = g.cx; P.cy = g.cy; P.cz = g.cz;
    P.gx0 = g.cx0; P.gy0 = g.cy0; P.gz0 = g.cz0;
    P.ginv_dx = 1.0 / g.cdx; P.ginv_dy = 1.0 / g.cdy; P.ginv_dz = 1.0 / g.cdz;
    P.zlut = c->n_lut > 0 ? c->d_zlut : nullptr;
    P.n_lut = c->n_lut;
    P.lut_z0 = c->lut_z0;
    P.lut_inv_h = c->lut_inv_h;
    P.m0 = c->d_m0;
    P.scen = c->d_scen;
    P.n_scen = g.n_scenarios;
    P.ctr_stride = g.n_scenarios;
    P.woff = c->any_woff ? c->d_woff : nullptr;
    P.conc_all = c->d_conc;
    P.ctr_all = c->d_ctr;
    P.dose_all = c->d_dose;
    P.dose_every = c->d_dose ? c->dose_every : 0;
    P.dose_mul = std::ldexp(1.0f, -c->dose_bits);
    P.blpair = c->kz_model == 1 ? c->d_blpair : nullptr;
    P.n_species = c->n_species;
    for (int j = 0; j < MAX_SPECIES; ++j) {
        P.chain_l[j] = (float)c->chain_l[j];
        for (int i = 0; i < MAX_SPECIES; ++i) P.chain_c[j][i] = (float)c->chain_c[j][i];
    }
    P.sp_conc_all = c->d_sp_conc;
    P.sp_dep_all = c->d_sp_dep;
    P.langevin = c->langevin;
    P.t_lagr = (float)c->t_lagr;
    P.kz_min = (float)c->kz_min;
    P.n_modes = c->d_mode_sc ? c->n_modes : 0;
    for (int m = 0; m < c->n_modes; ++m) {
        P.mode_fx[m] = (float)c->modes[m][0];
        P.mode_fy[m] = (float)c->modes[m][1];
        P.mode_om[m] = (float)c->modes[m][2];
        P.mode_eu[m] = (float)c->modes[m][3];
        P.mode_ev[m] = (float)c->modes[m][4];
    }
    for (size_t k = 0; k < c->mode_profile.size(); ++k) P.mode_prof[k] = (float)c->mode_profile[k];
    P.mode_sc = P.n_modes ? c->d_mode_sc : nullptr;
    P.slot_cap = c->cfg.max_particles;
    P.n_pair = std::max(1, g.n_met_t - 1);
    P.n_m0 = (int)c->d_m0_cap;
    P.err = c->d_err;
}

double emission_rate(const ScenHost &s, double dt, long long step)
{
    long long idx = (long long)std::floor((double)step * dt / s.q_dt);
    idx = std::max(0LL, std::min(idx, (long long)s.q.size() - 1));
    return s.q[(size_t)idx];
}

long long release_count(long long n, long long first, long long last, long long step)
{
    const long long S = last - first, j = step - first;
    if (j < 0 || j >= S) return 0;
    return ((j + 1) * n + S - 1) / S - (j * n + S - 1) / S;
}

lpm_status upload_tables(lpm_ctx *c)
{
    if (!c->tables_dirty) return LPM_OK;
    std::vector<float> m0;
    std::vector<ScenDev> sd(c->scen.size());
    const size_t nt = (size_t)c->cfg.n_met_t;
    std::vector<float2> woff(c->scen.size() * nt, make_float2(0.f, 0.f));
    c->any_woff = false;
    for (size_t s = 0; s < c->scen.size(); ++s) {
        const ScenHost &h = c->scen[s];
        ScenDev &d = sd[s];
        std::memset(&d, 0, sizeof d);
        d.src_x = (float)h.src_x; d.src_y = (float)h.src_y; d.src_z = (float)h.src_z;
        d.scale = pow2f(h.shift);
        d.first_slot = h.first_slot;
        d.n = h.n;
        d.id0 = h.id_base + h.part_first;
        d.rel_first = (int)h.rel_first;
        d.rel_last = (int)h.rel_last;
        d.m0_off = (int)m0.size();
        for (double v : h.m0) m0.push_back((float)v);
        if (!h.wind_offset.empty()) {
            for (size_t t = 0; t < nt; ++t)
                woff[s * nt + t] = make_float2(h.wind_offset[2 * t], h.wind_offset[2 * t + 1]);
            d.wind_offset = c->d_woff + s * nt;
            c->any_woff = true;
        }
        d.conc = c->d_conc + s * c->ncell();
        d.dep = c->d_dep + s * c->ndep();
        d.ctr = c->d_ctr + s;
        d.n_total = h.n_total;
        d.part_first = h.part_first;
    }
    if (m0.empty()) m0.push_back(0.f);
    std::vector<float> mq;
    std::vector<short> qi;
    for (size_t s = 0; s < c->scen.size(); ++s) {
        const ScenHost &h = c->scen[s];
        for (long long st = h.rel_first; st < h.rel_last; ++st) {
            const long long cnt = release_count(h.n_total, h.rel_first, h.rel_last, st);
            mq.push_back(cnt > 0 ? (float)(c->cfg.dt / (double)cnt) : 0.f);
            long long idx = (long long)std::floor((double)st * c->cfg.dt / h.q_dt);
            idx = std::max(0LL, std::min(idx, (long long)h.q.size() - 1));
            qi.push_back((short)idx);
        }
    }
    if (mq.empty()) { mq.push_back(0.f); qi.push_back(0); }
    if (m0.size() > c->d_m0_cap) {
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        for (void *p : {(void *)c->d_m0, (void *)c->d_mq, (void *)c->d_qi})
            if (p) cudaFree(p);
        c->d_m0 = nullptr;
        c->d_mq = nullptr;
        c->d_qi = nullptr;
        LPM_CUDA(c, cudaMalloc(&c->d_m0, m0.size() * sizeof(float)));
        LPM_CUDA(c, cudaMalloc(&c->d_mq, m0.size() * sizeof(float)));
        LPM_CUDA(c, cudaMalloc(&c->d_qi, m0.size() * sizeof(short)));
        c->d_m0_cap = m0.size();
    }
    // the stream may still read the old tables: order the copies on it
    LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    LPM_CUDA(c, cudaMemcpy(c->d_m0, m0.data(), m0.size() * sizeof(float), cudaMemcpyHostToDevice));
    LPM_CUDA(c, cudaMemcpy(c->d_mq, mq.data(), mq.size() * sizeof(float), cudaMemcpyHostToDevice));
    LPM_CUDA(c, cudaMemcpy(c->d_qi, qi.data(), qi.size() * sizeof(short), cudaMemcpyHostToDevice));
    LPM_CUDA(c, cudaMemcpy(c->d_scen, sd.data(), sd.size() * sizeof(ScenDev), cudaMemcpyHostToDevice));
    LPM_CUDA(c, cudaMemcpy(c->d_woff, woff.data(), woff.size() * sizeof(float2), cudaMemcpyHostToDevice));
    if (c->n_modes > 0) {
        std::vector<float> rows(c->scen.size() * 8, 0.0f);
        for (size_t s = 0; s < c->scen.size(); ++s)
            for (int m = 0; m < c->n_modes; ++m) {
                rows[s * 8 + (size_t)m] = (float)c->scen[s].mode_phase[m];
                rows[s * 8 + 4 + (size_t)m] = (float)c->scen[s].mode_amp[m];
            }
        if (!c->d_mode_sc)
            LPM_CUDA(c, cudaMalloc(&c->d_mode_sc, rows.size() * sizeof(float)));
        LPM_CUDA(c, cudaMemcpy(c->d_mode_sc, rows.data(), rows.size() * sizeof(float),
                               cudaMemcpyHostToDevice));
    }
    c->tables_dirty = false;
    c->params_version++;
    drop_graphs(c);
    return LPM_OK;
}

lpm_status check_device_error(lpm_ctx *c)
{
    unsigned int e = 0;
    LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->copy_stream) LPM_CUDA(c, cudaStreamSynchronize(c->copy_stream));
    LPM_CUDA(c, cudaMemcpy(&e, c->d_err, sizeof e, cudaMemcpyDeviceToHost));
    if (e & ERR_NAN) return fail(c, LPM_E_NUMERIC, "a particle position became non-finite");
    if (e & ERR_INDEX) return fail(c, LPM_E_CUDA, "a grid index fell outside its array");
    if (e & ERR_TIMEOUT) return fail(c, LPM_E_TIMEOUT, "a bounded device loop hit its limit");
    return LPM_OK;
}

// Initial mass per release step from the emission series (Sec. 3.2: masses assigned a
// priori from the emission profile and the particle budget) and the fixed-point scale.
lpm_status assign_masses(lpm_ctx *c, ScenHost &h)
{
    h.m0.assign((size_t)(h.rel_last - h.rel_first), 0.0);
    h.total_mass = 0.0;
    for (long long s = h.rel_first; s < h.rel_last; ++s) {
        const long long cnt = release_count(h.n_total, h.rel_first, h.rel_last, s);
        if (cnt <= 0) continue;
        const double rate = emission_rate(h, c->cfg.dt, s);
        h.m0[(size_t)(s - h.rel_first)] = rate * c->cfg.dt / (double)cnt;
        h.total_mass += rate * c->cfg.dt;
    }
    int e = 0;
    if (h.total_mass > 0) std::frexp(h.total_mass, &e);
    h.shift = h.total_mass > 0 ? 61 - e : 0;
    if (h.shift > 120 || h.shift < -120)
        return fail(c, LPM_E_INVALID, "total mass %g outside the fixed-point range", h.total_mass);
    return LPM_OK;
}

// Particles of a scenario's held range that leave before step k1.
long long released_before(const ScenHost &h, long long k1)
{
    const long long S = h.rel_last - h.rel_first;
    long long upto;                  // particles p < upto of the whole release
    if (k1 <= h.rel_first) upto = 0;
    else if (k1 >= h.rel_last) upto = h.n_total;
    else upto = ((k1 - h.rel_first) * h.n_total + S - 1) / S;
    return std::max(0LL, std::min(upto - h.part_first, h.n));
}

// Tile table (see lpm_ctx::tiles). A segment [k, e) after the sort at sorted_upto runs
// the tiles from the interval of sorted_upto up to the last tile whose first particle
// leaves before e; a sort at a multiple of E takes the tiles of the intervals since the
// previous sort. Tiles never straddle an interval, so no particle is in both sets.
lpm_status build_tiles(lpm_ctx *c)
{
    const int T = c->block * c->ppt;
    const long long NS = std::max<long long>(1, c->cfg.n_steps);
    const long long E = c->sort_every > 0 ? c->sort_every : NS;
    const long long n_int = (NS + E - 1) / E;
    c->tiles.clear();
    c->tile_sp.clear();
    c->int_lo.assign((size_t)n_int + 1, 0);
    std::vector<std::pair<long long, Tile>> items;
    for (long long j = 0; j < n_int; ++j) {
        c->int_lo[(size_t)j] = (int)c->tiles.size();
        items.clear();
        for (size_t s = 0; s < c->scen.size(); ++s) {
            const ScenHost &h = c->scen[s];
            const long long S = h.rel_last - h.rel_first;
            const long long a = released_before(h, j * E), b = released_before(h, (j + 1) * E);
            for (long long p = a; p < b; p += T) {
                Tile t;
                t.scen = (int)s;
                t.first = h.first_slot + p;
                t.count = (int)std::min<long long>(T, b - p);
                const long long sp = h.rel_first + ((h.part_first + p) * S) / h.n_total;
                items.push_back({sp, t});
            }
        }
        std::stable_sort(items.begin(), items.end(),
                         [](const auto &x, const auto &y) { return x.first < y.first; });
        for (auto &it : items) {
            c->tiles.push_back(it.second);
            c->tile_sp.push_back(it.first);
        }
    }
    c->int_lo[(size_t)n_int] = (int)c->tiles.size();
    c->tiles_E = E;
    LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (c->tiles.size() > c->d_tiles_cap || !c->d_tiles) {
        if (c->d_tiles) cudaFree(c->d_tiles);
        c->d_tiles = nullptr;
        LPM_CUDA(c, cudaMalloc(&c->d_tiles, std::max<size_t>(1, c->tiles.size()) * sizeof(Tile)));
        c->d_tiles_cap = std::max<size_t>(1, c->tiles.size());
    }
    if (!c->tiles.empty())
        LPM_CUDA(c, cudaMemcpy(c->d_tiles, c->tiles.data(), c->tiles.size() * sizeof(Tile),
                               cudaMemcpyHostToDevice));
    c->tiles_valid = true;
    drop_graphs(c);
    return LPM_OK;
}

// Index of the first tile whose first particle leaves at or after step e.
int tiles_before(const lpm_ctx *c, long long e)
{
    if (e <= 0 || c->tiles.empty()) return 0;
    const long long n_int = (long long)c->int_lo.size() - 1;
    const long long j = std::min((e - 1) / c->tiles_E, n_int - 1);
    const auto lo = c->tile_sp.begin() + c->int_lo[(size_t)j];
    const auto hi = c->tile_sp.begin() + c->int_lo[(size_t)j + 1];
    return (int)(std::lower_bound(lo, hi, e) - c->tile_sp.begin());
}

// Held particles (all scenarios) that leave before step k.
long long released_total(const lpm_ctx *c, long long k)
{
    long long n = 0;
    for (const ScenHost &h : c->scen) n += released_before(h, k);
    return n;
}

lpm_status ensure_sort_buffers(lpm_ctx *c, size_t keys_need)
{
    // allocate whatever is still missing (an earlier call may have stopped at a failure)
    const size_t n = (size_t)c->cfg.max_particles;
    const size_t nb = (size_t)sort_key_range(c->cfg.nx, c->cfg.ny, c->cfg.nz) + 1;
    const size_t ntiles = (nb + 1023) / 1024;
    auto need = [&](auto *&p, size_t bytes) -> cudaError_t {
        if (p) return cudaSuccess;
        drop_graphs(c);                      // graphs hold the buffers' addresses
        return cudaMalloc(&p, bytes);
    };
    for (int b = 0; b < 2; ++b) {
        LPM_CUDA(c, need(c->d_sorted[b], n * sizeof(float4)));
        LPM_CUDA(c, need(c->d_pidx[b], n * sizeof(unsigned int)));
    }
    if (!c->d_slot_of) {
        LPM_CUDA(c, need(c->d_slot_of, n * sizeof(unsigned int)));
        LPM_CUDA(c, cudaMemsetAsync(c->d_slot_of, 0xff, n * sizeof(unsigned int), c->stream));
    }
    LPM_CUDA(c, need(c->d_hist, nb * sizeof(unsigned int)));
    LPM_CUDA(c, need(c->d_bsums, ntiles * sizeof(unsigned int)));
    if (!c->d_live) {
        LPM_CUDA(c, need(c->d_live, 4 * sizeof(unsigned int)));
        LPM_CUDA(c, cudaMemsetAsync(c->d_live, 0, 4 * sizeof(unsigned int), c->stream));
    }
    LPM_CUDA(c, need(c->d_grave, n * sizeof(float4)));
    LPM_CUDA(c, need(c->d_grave_home, n * sizeof(unsigned int)));
    if (!c->d_grave_n) {
        LPM_CUDA(c, need(c->d_grave_n, sizeof(unsigned int)));
        LPM_CUDA(c, cudaMemsetAsync(c->d_grave_n, 0, sizeof(unsigned int), c->stream));
    }
    if (keys_need > c->keys_cap) {
        drop_graphs(c);
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        if (c->d_keys) cudaFree(c->d_keys);
        c->d_keys = nullptr;
        c->keys_cap = 0;
        LPM_CUDA(c, cudaMalloc(&c->d_keys, keys_need * sizeof(unsigned int)));
        c->keys_cap = keys_need;
    }
    return LPM_OK;
}

// The slot map (home slot -> sorted slot, dead entry or home) for the read-back paths: the
// sorts leave it to be rebuilt here, from the sorted and dead sets, when it is asked for.
lpm_status ensure_slot_map(lpm_ctx *c)
{
    if (!c->slot_map_stale || !c->d_slot_of) return LPM_OK;
    LPM_CUDA(c, launch_slot_map(c->stream, c->d_pidx[c->cur], c->d_live, c->d_grave_home,
                                c->d_grave_n, c->d_slot_of, (long long)c->cfg.max_particles,
                                c->d_err));
    c->n_launches++;
    c->slot_map_stale = false;
    return LPM_OK;
}

// Empties the sorted set: every particle back to its home slot.
lpm_status clear_sort_state(lpm_ctx *c, bool move_back)
{
    if (c->d_sorted[0]) {
        if (move_back && c->sorted_upto > 0) {
            lpm_status st = ensure_slot_map(c);
            if (st != LPM_OK) return st;
        }
        if (move_back && c->sorted_upto > 0)
            LPM_CUDA(c, launch_unsort(c->stream, c->d_state, c->d_sorted[c->cur], c->d_slot_of,
                                      c->d_grave, c->n_slots_used,
                                      c->langevin ? c->d_w_home : nullptr,
                                      c->langevin ? c->d_w_sorted[c->cur] : nullptr));
        else
            LPM_CUDA(c, cudaMemsetAsync(c->d_slot_of, 0xff,
                                        (size_t)c->cfg.max_particles * sizeof(unsigned int),
                                        c->stream));
        LPM_CUDA(c, cudaMemsetAsync(c->d_live, 0, 4 * sizeof(unsigned int), c->stream));
        LPM_CUDA(c, cudaMemsetAsync(c->d_grave_n, 0, sizeof(unsigned int), c->stream));
        c->n_launches++;
    }
    c->slot_map_stale = false;               // every slot is home again
    c->sorted_upto = 0;
    c->cur = 0;
    return LPM_OK;
}

cudaEvent_t next_event(lpm_ctx *c)
{
    if (c->ev_used == c->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        c->ev_pool.push_back(e);
    }
    return c->ev_pool[c->ev_used++];
}

// Adds the elapsed time of recorded (start, stop) pairs to adv_ms (synchronises).
lpm_status collect_events(lpm_ctx *c)
{
    if (c->ev_used == 0) return LPM_OK;
    LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
        float ms = 0.f;
        LPM_CUDA(c, cudaEventElapsedTime(&ms, c->ev_pool[i], c->ev_pool[i + 1]));
        c->adv_ms += ms;
    }
    c->ev_used = 0;
    return LPM_OK;
}

lpm_status read_counters(lpm_ctx *c, int scenario, unsigned long long v[N_COUNTERS])
{
    const size_t ns = (size_t)c->cfg.n_scenarios;
    for (int i = 0; i < N_COUNTERS; ++i)
        LPM_CUDA(c, cudaMemcpy(v + i, c->d_ctr + i * ns + scenario, sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost));
    return LPM_OK;
}

void drop_graphs(lpm_ctx *c)
{
    for (auto &g : c->graphs) cudaGraphExecDestroy(g.exec);
    c->graphs.clear();
}

}  // namespace

namespace lpm {
// Records the text lpm_last_error(NULL) returns (entry points without a context).
void set_global_error(const char *msg) { g_create_error = msg; }
}  // namespace lpm

// =====================================================================================
// C ABI
// =====================================================================================
extern "C" {

lpm_status lpm_create(const lpm_config *cfg, void *cuda_stream, lpm_ctx **out)
{
    if (!out) return fail(nullptr, LPM_E_INVALID, "out is NULL");
    *out = nullptr;
    lpm_status st = validate(cfg);
    if (st != LPM_OK) return st;
    lpm_ctx *c = new (std::nothrow) lpm_ctx();
    if (!c) return fail(nullptr, LPM_E_OOM, "host allocation failed");
    c->cfg = *cfg;
    c->zlev.assign(cfg->z_levels, cfg->z_levels + cfg->nz);
    c->cfg.z_levels = nullptr;
    c->stream = (cudaStream_t)cuda_stream;
    c->met_set.assign((size_t)cfg->n_met_t, 0);
    c->scen.resize((size_t)cfg->n_scenarios);
    c->scen[0].src_x = cfg->src_x;
    c->scen[0].src_y = cfg->src_y;
    c->scen[0].src_z = cfg->src_z;
    auto bail = [&](lpm_status s) {
        g_create_error = c->err;
        lpm_destroy(c);
        return s;
    };
#define CREATE_CUDA(call)                                                                  \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess) {                                                           \
            (void)cudaGetLastError();                                                      \
            fail(c, e_ == cudaErrorMemoryAllocation ? LPM_E_OOM : LPM_E_CUDA, "%s: %s",   \
                 #call, cudaGetErrorString(e_));                                           \
            return bail(e_ == cudaErrorMemoryAllocation ? LPM_E_OOM : LPM_E_CUDA);         \
        }                                                                                  \
    } while (0)
    CREATE_CUDA(cudaGetDevice(&c->device));
    CREATE_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, c->device));
    const size_t nodes = (size_t)cfg->nx * cfg->ny * cfg->nz;
    const size_t ns = (size_t)cfg->n_scenarios;
    const size_t n_pair = (size_t)std::max(1, cfg->n_met_t - 1);
    CREATE_CUDA(cudaMalloc(&c->d_uvwk, nodes * cfg->n_met_t * sizeof(float4)));
    CREATE_CUDA(cudaMalloc(&c->d_pair, nodes * n_pair * 2 * sizeof(float4)));
    if (cfg->kh_uniform < 0) {
        CREATE_CUDA(cudaMalloc(&c->d_kh, nodes * cfg->n_met_t * sizeof(float)));
        CREATE_CUDA(cudaMalloc(&c->d_khpair, nodes * n_pair * sizeof(float2)));
    }
    CREATE_CUDA(cudaMalloc(&c->d_rain, (size_t)cfg->nx * cfg->ny * cfg->n_met_t));
    CREATE_CUDA(cudaMemsetAsync(c->d_rain, 0, (size_t)cfg->nx * cfg->ny * cfg->n_met_t, c->stream));
    CREATE_CUDA(cudaMalloc(&c->d_state, (size_t)cfg->max_particles * sizeof(float4)));
    CREATE_CUDA(cudaMalloc(&c->d_conc, ns * c->ncell() * sizeof(unsigned long long)));
    CREATE_CUDA(cudaMalloc(&c->d_dep, ns * c->ndep() * sizeof(unsigned long long)));
    CREATE_CUDA(cudaMalloc(&c->d_ctr, ns * N_COUNTERS * sizeof(unsigned long long)));
    CREATE_CUDA(cudaMalloc(&c->d_err, sizeof(unsigned int)));
    CREATE_CUDA(cudaMalloc(&c->d_queue, sizeof(unsigned int)));
    CREATE_CUDA(cudaMalloc(&c->d_scen, ns * sizeof(ScenDev)));
    CREATE_CUDA(cudaMalloc(&c->d_woff, ns * cfg->n_met_t * sizeof(float2)));
    CREATE_CUDA(cudaMemsetAsync(c->d_conc, 0, ns * c->ncell() * sizeof(unsigned long long), c->stream));
    CREATE_CUDA(cudaMemsetAsync(c->d_dep, 0, ns * c->ndep() * sizeof(unsigned long long), c->stream));
    CREATE_CUDA(cudaMemsetAsync(c->d_ctr, 0, ns * N_COUNTERS * sizeof(unsigned long long), c->stream));
    CREATE_CUDA(cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), c->stream));
    {
        // vertical lookup table: bins of the smallest level spacing / 1.2, each holding the
        // cell 0.05 bin below its lower edge (the kernel then corrects it by at most one with
        // one comparison: the 1.05 bins from that point to the bin's top hold at most one
        // level), in the FP32 arithmetic the kernel uses to pick a bin; fewer, wider bins
        // spread a warp's lookups over fewer shared-memory words
        std::vector<float> zf(cfg->nz);
        for (int k = 0; k < cfg->nz; ++k) zf[k] = (float)cfg->z_levels[k];
        double min_sp = 1e300;
        for (int k = 0; k + 1 < cfg->nz; ++k) min_sp = std::min(min_sp, (double)zf[k + 1] - zf[k]);
        const double span = (double)zf[cfg->nz - 1] - zf[0];
        const double n_need = min_sp > 0 ? std::ceil(span / (min_sp / 1.2)) + 1 : 1e300;
        if (n_need <= MAX_LUT) {
            c->n_lut = (int)n_need;
            c->lut_z0 = zf[0];
            c->lut_inv_h = (float)((c->n_lut - 1) / span);
            std::vector<unsigned char> lut((size_t)c->n_lut);
            for (int b = 0; b < c->n_lut; ++b) {
                const double zb = (double)zf[0] + (b - 0.05) / (double)c->lut_inv_h;
                int k = 0;
                for (int m = 0; m < cfg->nz; ++m)
                    if ((double)zf[m] <= zb) k = m;
                lut[(size_t)b] = (unsigned char)std::min(k, cfg->nz - 2);
            }
            CREATE_CUDA(cudaMalloc(&c->d_zlut, lut.size()));
            CREATE_CUDA(cudaMemcpy(c->d_zlut, lut.data(), lut.size(), cudaMemcpyHostToDevice));
        }
    }
    CREATE_CUDA(cudaStreamSynchronize(c->stream));
#undef CREATE_CUDA
    *out = c;
    return LPM_OK;
}

void lpm_destroy(lpm_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    void *ptrs[] = {c->d_uvwk, c->d_kh, c->d_pair, c->d_khpair, c->d_rain, c->d_state, c->d_conc, c->d_dep, c->d_ctr,
                    c->d_err, c->d_queue, c->d_m0, c->d_scen, c->d_woff, c->d_tiles,
                    c->d_zlut, c->d_mq, c->d_qi, c->d_ckpt, c->d_rec, c->d_rC, c->d_rw,
                    c->d_rgrad, c->d_adj_tiles, c->d_sorted[0], c->d_sorted[1], c->d_pidx[0],
                    c->d_pidx[1], c->d_slot_of, c->d_keys, c->d_hist, c->d_bsums, c->d_live,
                    c->d_grave, c->d_grave_n, c->d_grave_home, c->d_dose, c->d_bl, c->d_blpair,
                    c->d_sp_conc, c->d_sp_dep, c->d_w_home, c->d_w_sorted[0],
                    c->d_w_sorted[1], c->d_traj, c->d_fin, c->d_traj_tile, c->d_conv,
                    c->d_rbin_off, c->d_rbin_idx, c->d_mode_sc};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    {
        lpm_ctx::AdjSorted &S = c->as;
        void *aps[] = {S.d_tiles, S.ord, S.live, S.keys, S.hist, S.bsums, S.meta, S.slot_of,
                       S.grave_n, S.st[0], S.st[1], S.home, S.mu, S.grave};
        for (void *p : aps)
            if (p) cudaFree(p);
    }
    if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (cudaEvent_t e : c->ev_pair)
        if (e) cudaEventDestroy(e);
    if (c->ev_main) cudaEventDestroy(c->ev_main);
    if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
    if (c->adj_stream) cudaStreamSynchronize(c->adj_stream);
    for (cudaEvent_t e : c->ev_adj)
        if (e) cudaEventDestroy(e);
    if (c->adj_stream) cudaStreamDestroy(c->adj_stream);
    drop_graphs(c);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

const char *lpm_last_error(const lpm_ctx *c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

namespace {

bool is_pinned_host(const void *p)
{
    if (!p) return true;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

}  // namespace

lpm_status lpm_set_met(lpm_ctx *c, int t_index, const float *uvwk, const float *kh,
                       const uint8_t *rain, int on_device)
{
    if (!c) return LPM_E_INVALID;
    const lpm_config &g = c->cfg;
    if (t_index < 0 || t_index >= g.n_met_t)
        return fail(c, LPM_E_INVALID, "t_index %d outside [0, %d)", t_index, g.n_met_t);
    if (!uvwk) return fail(c, LPM_E_INVALID, "uvwk is NULL");
    if ((g.kh_uniform < 0) != (kh != nullptr))
        return fail(c, LPM_E_INVALID, "kh must be given iff kh_uniform < 0");
    const size_t nodes = (size_t)g.nx * g.ny * g.nz;
    const size_t cols = (size_t)g.nx * g.ny;
    const bool async = !on_device && is_pinned_host(uvwk) && is_pinned_host(kh) &&
                       is_pinned_host(rain);
    cudaStream_t s = c->stream;
    if (async) {
        // copy after everything already enqueued (earlier runs may still read the slabs)
        if (!c->copy_stream)
            LPM_CUDA(c, cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
        if (!c->ev_main) LPM_CUDA(c, cudaEventCreateWithFlags(&c->ev_main, cudaEventDisableTiming));
        if (c->ev_pair.empty()) {
            c->ev_pair.assign((size_t)std::max(1, g.n_met_t - 1), nullptr);
            c->pair_pending.assign(c->ev_pair.size(), 0);
        }
        LPM_CUDA(c, cudaEventRecord(c->ev_main, c->stream));
        LPM_CUDA(c, cudaStreamWaitEvent(c->copy_stream, c->ev_main, 0));
        s = c->copy_stream;
    } else if (c->copy_stream) {
        LPM_CUDA(c, cudaStreamSynchronize(c->copy_stream));   // no copy of ours in flight
    }
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    LPM_CUDA(c, cudaMemcpyAsync(c->d_uvwk + nodes * t_index, uvwk, nodes * sizeof(float4), kind, s));
    if (kh)
        LPM_CUDA(c, cudaMemcpyAsync(c->d_kh + nodes * t_index, kh, nodes * sizeof(float), kind, s));
    if (rain) {
        LPM_CUDA(c, cudaMemcpyAsync(c->d_rain + cols * t_index, rain, cols, kind, s));
        if (!c->any_rain) drop_graphs(c);    // captured launches baked in "no rain"
        c->any_rain = true;
    } else {
        LPM_CUDA(c, cudaMemsetAsync(c->d_rain + cols * t_index, 0, cols, s));
    }
    c->met_set[(size_t)t_index] = 1;
    // time pairs (h, h+1) that this slab completes
    for (int h = t_index - 1; h <= t_index; ++h) {
        const int h1 = g.n_met_t > 1 ? h + 1 : h;
        if (h < 0 || h1 > g.n_met_t - 1 || (g.n_met_t > 1 && h > g.n_met_t - 2)) continue;
        if (!c->met_set[(size_t)h] || !c->met_set[(size_t)h1]) continue;
        LPM_CUDA(c, launch_pack(s, c->d_uvwk + nodes * h, c->d_uvwk + nodes * h1,
                                c->d_kh ? c->d_kh + nodes * h : nullptr,
                                c->d_kh ? c->d_kh + nodes * h1 : nullptr,
                                c->d_pair + nodes * 2 * h, c->d_khpair ? c->d_khpair + nodes * h : nullptr,
                                g.nx, g.ny, g.nz));
        c->n_launches++;
        if (async) {
            if (!c->ev_pair[(size_t)h])
                LPM_CUDA(c, cudaEventCreateWithFlags(&c->ev_pair[(size_t)h], cudaEventDisableTiming));
            LPM_CUDA(c, cudaEventRecord(c->ev_pair[(size_t)h], c->copy_stream));
            c->pair_pending[(size_t)h] = 1;
        }
    }
    // pageable host sources must be consumed before returning (the caller owns them)
    if (!on_device && !async) LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LPM_OK;
}

lpm_status lpm_set_source(lpm_ctx *c, int scenario, double x, double y, double z,
                          const float *wind_offset)
{
    if (!c) return LPM_E_INVALID;
    if (scenario < 0 || scenario >= c->cfg.n_scenarios)
        return fail(c, LPM_E_INVALID, "scenario %d outside [0, %d)", scenario, c->cfg.n_scenarios);
    if (!is_finite(x) || !is_finite(y) || !is_finite(z))
        return fail(c, LPM_E_INVALID, "source must be finite");
    ScenHost &h = c->scen[(size_t)scenario];
    std::vector<float> wo;
    if (wind_offset) {
        wo.assign(wind_offset, wind_offset + 2 * (size_t)c->cfg.n_met_t);
        for (float v : wo)
            if (!std::isfinite(v)) return fail(c, LPM_E_INVALID, "wind offset not finite");
    }
    if (h.src_x == x && h.src_y == y && h.src_z == z && h.wind_offset == wo) return LPM_OK;
    h.src_x = x; h.src_y = y; h.src_z = z;
    h.wind_offset = wo;
    c->tables_dirty = true;
    return LPM_OK;
}

lpm_status lpm_set_modes(lpm_ctx *c, int n_modes, const double *modes, const double *profile)
{
    if (!c) return LPM_E_INVALID;
    if (n_modes < 0 || n_modes > MAX_MODES)
        return fail(c, LPM_E_INVALID, "n_modes=%d outside [0, %d]", n_modes, MAX_MODES);
    if (n_modes > 0 && (!modes || !profile))
        return fail(c, LPM_E_INVALID, "modes and profile are required");
    for (int i = 0; i < 5 * n_modes; ++i)
        if (!is_finite(modes[i])) return fail(c, LPM_E_INVALID, "mode parameters not finite");
    for (int k = 0; n_modes > 0 && k < c->cfg.nz; ++k)
        if (!is_finite(profile[k])) return fail(c, LPM_E_INVALID, "mode profile not finite");
    c->n_modes = n_modes;
    std::memset(c->modes, 0, sizeof c->modes);
    for (int m = 0; m < n_modes; ++m)
        for (int q = 0; q < 5; ++q) c->modes[m][q] = modes[5 * m + q];
    if (n_modes > 0) c->mode_profile.assign(profile, profile + c->cfg.nz);
    else c->mode_profile.clear();
    c->tables_dirty = true;
    c->adj_sig.clear();
    drop_graphs(c);                          // the graphs hold the step parameters
    return LPM_OK;
}

lpm_status lpm_set_mode_phases(lpm_ctx *c, int scenario, const double *phase, const double *amp)
{
    if (!c) return LPM_E_INVALID;
    if (scenario < 0 || scenario >= c->cfg.n_scenarios)
        return fail(c, LPM_E_INVALID, "scenario %d outside [0, %d)", scenario, c->cfg.n_scenarios);
    if (c->n_modes > 0 && (!phase || !amp))
        return fail(c, LPM_E_INVALID, "phase and amp are required");
    for (int m = 0; m < c->n_modes; ++m)
        if (!is_finite(phase[m]) || !is_finite(amp[m]))
            return fail(c, LPM_E_INVALID, "mode phases and amplitudes must be finite");
    ScenHost &h = c->scen[(size_t)scenario];
    for (int m = 0; m < MAX_MODES; ++m) {
        h.mode_phase[m] = m < c->n_modes ? phase[m] : 0.0;
        h.mode_amp[m] = m < c->n_modes ? amp[m] : 0.0;
    }
    c->tables_dirty = true;
    c->adj_sig.clear();
    return LPM_OK;
}

lpm_status lpm_release_range(lpm_ctx *c, int scenario, int64_t n_total, int64_t first_particle,
                             int64_t count, const double *q, int n_q, double q_dt,
                             int64_t first, int64_t last, int64_t id_base)
{
    if (!c) return LPM_E_INVALID;
    NvtxRange nr("lpm_release");
    if (scenario != c->n_released)
        return fail(c, LPM_E_STATE, "scenarios must be released once each, in order (next is %d)",
                    c->n_released);
    if (scenario >= c->cfg.n_scenarios) return fail(c, LPM_E_INVALID, "scenario out of range");
    if (n_total < 1 || !q || n_q < 1 || !(q_dt > 0) || first < 0 || last <= first ||
        last > c->cfg.n_steps)
        return fail(c, LPM_E_INVALID, "invalid release (n=%lld, n_q=%d, steps [%lld, %lld))",
                    (long long)n_total, n_q, (long long)first, (long long)last);
    if (first_particle < 0 || count < 1 || first_particle + count > n_total || id_base < 0)
        return fail(c, LPM_E_INVALID, "particle range [%lld, %lld) outside [0, %lld)",
                    (long long)first_particle, (long long)(first_particle + count),
                    (long long)n_total);
    if (c->n_slots_used + count > c->cfg.max_particles)
        return fail(c, LPM_E_INVALID, "release exceeds max_particles");
    if (c->k > first)
        return fail(c, LPM_E_STATE, "release starts before the current step");
    for (int i = 0; i < n_q; ++i)
        if (!is_finite(q[i]) || q[i] < 0) return fail(c, LPM_E_INVALID, "emission rates must be >= 0");
    ScenHost &h = c->scen[(size_t)scenario];
    h.first_slot = c->n_slots_used;
    h.n = count;
    h.n_total = n_total;
    h.part_first = first_particle;
    h.id_base = id_base;
    h.rel_first = first;
    h.rel_last = last;
    h.q.assign(q, q + n_q);
    h.q_dt = q_dt;
    lpm_status mst = assign_masses(c, h);
    if (mst != LPM_OK) return mst;
    h.released = true;
    c->n_slots_used += count;
    c->n_ids_used = std::max<long long>(c->n_ids_used, id_base + n_total);
    c->n_released++;
    c->tables_dirty = true;
    c->tiles_valid = false;
    LPM_CUDA(c, launch_release(c->stream, c->d_state, h.first_slot, h.n, h.part_first, h.n_total,
                               (int)first, (int)(last - first), (float)h.src_x, (float)h.src_y,
                               (float)h.src_z));
    c->n_launches++;
    return LPM_OK;
}

lpm_status lpm_release(lpm_ctx *c, int scenario, int64_t n, const double *q, int n_q, double q_dt,
                       int64_t first, int64_t last)
{
    if (!c) return LPM_E_INVALID;
    return lpm_release_range(c, scenario, n, 0, n, q, n_q, q_dt, first, last, c->n_ids_used);
}

lpm_status lpm_reset(lpm_ctx *c)
{
    if (!c) return LPM_E_INVALID;
    NvtxRange nr("lpm_reset");
    const size_t ns = (size_t)c->cfg.n_scenarios;
    LPM_CUDA(c, cudaMemsetAsync(c->d_conc, 0, ns * c->ncell() * sizeof(unsigned long long), c->stream));
    LPM_CUDA(c, cudaMemsetAsync(c->d_dep, 0, ns * c->ndep() * sizeof(unsigned long long), c->stream));
    LPM_CUDA(c, cudaMemsetAsync(c->d_ctr, 0, ns * N_COUNTERS * sizeof(unsigned long long), c->stream));
    LPM_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), c->stream));
    lpm_status st = upload_tables(c);
    if (st != LPM_OK) return st;
    StepParams P;
    fill_params(c, P);
    LPM_CUDA(c, launch_release_all(c->stream, P, c->d_state, c->n_slots_used));
    c->n_launches++;
    st = clear_sort_state(c, false);
    if (st != LPM_OK) return st;
    if (c->d_dose)
        LPM_CUDA(c, cudaMemsetAsync(c->d_dose, 0, ns * c->ncell() * sizeof(unsigned long long),
                                    c->stream));
    if (c->n_species > 1) {
        const size_t nd = (size_t)(c->n_species - 1) * ns;
        LPM_CUDA(c, cudaMemsetAsync(c->d_sp_conc, 0, nd * c->ncell() * 8, c->stream));
        LPM_CUDA(c, cudaMemsetAsync(c->d_sp_dep, 0, nd * c->ndep() * 8, c->stream));
    }
    if (c->d_w_home)
        LPM_CUDA(c, cudaMemsetAsync(c->d_w_home, 0, (size_t)c->cfg.max_particles * sizeof(float),
                                    c->stream));
    c->k = 0;
    c->n_bins = 0;
    c->n_dose = 0;
    return LPM_OK;
}

lpm_status lpm_set_profiling(lpm_ctx *c, int on)
{
    if (!c) return LPM_E_INVALID;
    lpm_status st = collect_events(c);
    if (st != LPM_OK) return st;
    c->profiling = on != 0;
    return LPM_OK;
}

lpm_status lpm_stats(lpm_ctx *c, int64_t *launches, int64_t *advance_launches,
                     double *advance_ms)
{
    if (!c) return LPM_E_INVALID;
    lpm_status st = collect_events(c);
    if (st != LPM_OK) return st;
    if (launches) *launches = c->n_launches;
    if (advance_launches) *advance_launches = c->n_adv_launches;
    if (advance_ms) *advance_ms = c->adv_ms;
    c->n_launches = 0;
    c->n_adv_launches = 0;
    c->adv_ms = 0.0;
    return LPM_OK;
}

lpm_status lpm_set_launch(lpm_ctx *c, int block, int ppt, int occupancy)
{
    if (!c) return LPM_E_INVALID;
    if (!(block == 128 || block == 256 || block == 512) || !(ppt == 1 || ppt == 2 || ppt == 4) ||
        occupancy < 0 || occupancy > 2)
        return fail(c, LPM_E_INVALID, "launch shape %d x %d (occupancy %d) not supported", block, ppt,
                    occupancy);
    c->block = block;
    c->ppt = ppt;
    c->occ = occupancy;
    c->tiles_valid = false;
    drop_graphs(c);
    return LPM_OK;
}

namespace {

// Makes stream s wait for the weather pairs that steps [k0, k1) read and that a
// page-locked upload may still be writing.
lpm_status wait_met_pairs(lpm_ctx *c, cudaStream_t s, long long k0, long long k1)
{
    if (!c->copy_stream || k1 <= k0) return LPM_OK;
    const lpm_config &g = c->cfg;
    const long long n_pair = (long long)c->pair_pending.size();
    long long h_a = (long long)std::floor(((double)k0 * g.dt - g.met_t0) / g.met_dt);
    long long h_b = (long long)std::floor(((double)(k1 - 1) * g.dt - g.met_t0) / g.met_dt);
    h_a = std::max(0LL, std::min(h_a, n_pair - 1));
    h_b = std::max(0LL, std::min(h_b, n_pair - 1));
    for (long long h = h_a; h <= h_b; ++h)
        if (c->pair_pending[(size_t)h]) LPM_CUDA(c, cudaStreamWaitEvent(s, c->ev_pair[(size_t)h], 0));
    return LPM_OK;
}

// One segment [k, e) of an lpm_step call: an optional sort at k, then one advance launch.
struct Segment {
    long long k, e;
    bool do_bin, sort, sort_has_a;
    long long sort_a_bound;            // live-count bound of the sorted set before the sort
    int sort_b_lo, sort_b_hi;          // tiles whose particles join the sorted set
    long long a_bound;                 // live-count bound of the sorted set during the launch
    int b_lo, b_hi;                    // tiles run from their home slots
};

// Issues the segments on stream s, starting from sort state (upto, cur); returns the
// kernels launched and leaves the final sort state in (upto, cur). `direct`: launched now
// (not captured), so advance launches are counted and, with profiling, timed.
lpm_status run_segments(lpm_ctx *c, const StepParams &P, const std::vector<Segment> &plan,
                        cudaStream_t s, long long &upto, int &cur, long long &kernels,
                        bool direct, int occ_blocks)
{
    const lpm_config &g = c->cfg;
    const bool batched = g.n_scenarios > 1;
    const int T = c->block * c->ppt;
    const size_t ns = (size_t)g.n_scenarios;
    bool keys_ready = false;                 // the previous launch wrote the sort's keys
    for (size_t gi = 0; gi < plan.size(); ++gi) {
        const Segment &sg = plan[gi];
        if (direct) {
            lpm_status ws = wait_met_pairs(c, s, sg.k, sg.e);
            if (ws != LPM_OK) return ws;
        }
        if (sg.do_bin) {
            LPM_CUDA(c, cudaMemsetAsync(c->d_conc, 0, ns * c->ncell() * sizeof(unsigned long long), s));
            LPM_CUDA(c, cudaMemsetAsync(c->d_ctr + (size_t)C_BIN_OUT * ns, 0,
                                        ns * sizeof(unsigned long long), s));
            if (c->n_species > 1) {
                LPM_CUDA(c, cudaMemsetAsync(c->d_sp_conc, 0, (size_t)(c->n_species - 1) * ns *
                                                                 c->ncell() * 8, s));
                LPM_CUDA(c, cudaMemsetAsync(c->d_ctr + (size_t)C_SP_OUT * ns, 0,
                                            (size_t)(c->n_species - 1) * ns * 8, s));
            }
        }
        if (sg.sort) {
            NvtxRange nr("lpm sort");
            SortSource in{};
            in.state_a = c->d_sorted[cur];
            in.pidx_a = c->d_pidx[cur];
            in.has_a = sg.sort_has_a;
            in.a_bound = sg.sort_a_bound;
            in.state_b = c->d_state;
            in.tiles = c->d_tiles;
            in.b_first = sg.sort_b_lo;
            in.n_b = sg.sort_b_hi - sg.sort_b_lo;
            in.T = T;
            in.w_a = c->langevin ? c->d_w_sorted[cur] : nullptr;
            in.w_b = c->langevin ? c->d_w_home : nullptr;
            in.keys_ready = keys_ready;
            SortBuffers out{};
            out.state_out = c->d_sorted[1 - cur];
            out.pidx_out = c->d_pidx[1 - cur];
            out.slot_of = nullptr;               // rebuilt on request (ensure_slot_map)
            out.grave_home = c->d_grave_home;
            out.keys = c->d_keys;
            out.hist = c->d_hist;
            out.block_sums = c->d_bsums;
            out.meta = c->d_live;
            out.grave = c->d_grave;
            out.grave_count = c->d_grave_n;
            out.w_out = c->langevin ? c->d_w_sorted[1 - cur] : nullptr;
            out.cap = c->cfg.max_particles;
            out.err = c->d_err;
            LPM_CUDA(c, launch_sort(s, P, in, out));
            c->slot_map_stale = true;
            cur = 1 - cur;
            upto = sg.k;
            kernels += keys_ready ? 6 : 7;
        }
        AdvanceLaunch L{};
        L.stream = s;
        L.params = &P;
        L.ranges.state_a = c->d_sorted[cur];
        L.ranges.a_live = c->d_live;
        L.ranges.pidx = c->d_pidx[cur];
        L.ranges.tiles_a = (int)((sg.a_bound + T - 1) / T);
        L.ranges.state_b = c->d_state;
        L.ranges.b_tiles = c->d_tiles;
        L.ranges.b_first = sg.b_lo;
        L.ranges.n_b = sg.b_hi - sg.b_lo;
        L.ranges.w_a = c->langevin ? c->d_w_sorted[cur] : nullptr;
        L.ranges.w_b = c->langevin ? c->d_w_home : nullptr;
        L.k0 = (int)sg.k;
        L.k1 = (int)sg.e;
        L.do_bin = sg.do_bin ? 1 : 0;
        L.block = c->block;
        L.ppt = c->ppt;
        L.occ = c->occ;
        L.mixed = batched;
        L.ext = P.dose_every > 0 || P.blpair != nullptr || P.n_species > 1 || P.langevin;
        L.modes = P.n_modes > 0;
        const int n_tiles = L.n_tiles();
        keys_ready = false;
        if (n_tiles <= 0) continue;
        // the next segment starts with a sort of exactly these particles: write its keys here
        // (one scenario: measured +0.9 %; the 256-scenario ensemble sorted every 30 steps:
        // +0.3 %)
        const Segment *nx = gi + 1 < plan.size() ? &plan[gi + 1] : nullptr;
        if (nx && nx->sort && nx->sort_b_lo == sg.b_lo && nx->sort_b_hi == sg.b_hi &&
            nx->sort_a_bound == (upto > 0 ? sg.a_bound : 0)) {
            const size_t nb = (size_t)sort_key_range(g.nx, g.ny, g.nz) + 1;
            LPM_CUDA(c, cudaMemsetAsync(c->d_hist, 0, nb * sizeof(unsigned int), s));
            L.ranges.keys = c->d_keys;
            L.ranges.hist = c->d_hist;
            keys_ready = true;
        }
        // persistent grid over an atomic tile queue (the plain run: measured +0.8 % against
        // a grid of all tiles, each block loading the level table once for many tiles)
        LPM_CUDA(c, cudaMemsetAsync(c->d_queue, 0, sizeof(unsigned int), s));
        L.queue = c->d_queue;
        L.grid = (unsigned)std::max(1, std::min(n_tiles, occ_blocks * c->sm_count));
        const bool timed = direct && c->profiling;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (timed) {
            e0 = next_event(c);
            e1 = next_event(c);
            if (!e0 || !e1) return fail(c, LPM_E_CUDA, "cudaEventCreate failed");
            LPM_CUDA(c, cudaEventRecord(e0, s));
        }
        {
            NvtxRange nr("lpm advance");
            LPM_CUDA(c, launch_advance(L));
        }
        if (timed) LPM_CUDA(c, cudaEventRecord(e1, s));
        if (direct) c->n_adv_launches++;
        kernels++;
    }
    return LPM_OK;
}

}  // namespace

lpm_status lpm_step(lpm_ctx *c, int64_t n)
{
    if (!c) return LPM_E_INVALID;
    NvtxRange nr("lpm_step");
    const lpm_config &g = c->cfg;
    if (n < 0) return fail(c, LPM_E_INVALID, "n must be >= 0");
    if (n == 0) return LPM_OK;
    if (c->n_released != g.n_scenarios)
        return fail(c, LPM_E_STATE, "%d of %d scenarios released", c->n_released, g.n_scenarios);
    if (c->k + n > g.n_steps)
        return fail(c, LPM_E_STATE, "stepping to %lld passes n_steps=%lld",
                    (long long)(c->k + n), (long long)g.n_steps);
    // met slabs touched by t in [t_k, t_{k+n-1}]
    {
        const double t_a = (double)c->k * g.dt, t_b = (double)(c->k + n - 1) * g.dt;
        long long h_a = (long long)std::floor((t_a - g.met_t0) / g.met_dt);
        long long h_b = (long long)std::floor((t_b - g.met_t0) / g.met_dt) + 1;
        h_a = std::max(0LL, std::min(h_a, (long long)g.n_met_t - 1));
        h_b = std::max(0LL, std::min(h_b, (long long)g.n_met_t - 1));
        for (long long h = h_a; h <= h_b; ++h) {
            if (!c->met_set[(size_t)h])
                return fail(c, LPM_E_STATE, "met slab %lld not set", h);
            if (c->kz_model == 1 && !c->bl_set[(size_t)h])
                return fail(c, LPM_E_STATE, "boundary-layer slab %lld not set", h);
        }
    }
    lpm_status st = LPM_OK;
    if (c->copy_stream && g.n_scenarios > 1) {
        // weather pairs still in flight from page-locked uploads: the graph of the call
        // waits for all those it reads (the plain form waits segment by segment)
        st = wait_met_pairs(c, c->stream, c->k, c->k + n);
        if (st != LPM_OK) return st;
    }
    const bool ext = (c->d_dose && c->dose_every > 0) || c->kz_model == 1 || c->n_species > 1 ||
                     c->langevin || c->n_modes > 0;
    if (ext && c->ppt != 1)
        return fail(c, LPM_E_INVALID, "dosage, K_z from Eq. 3, decay chains, the Langevin "
                                      "variant and perturbation modes run with 1 particle per "
                                      "thread");
    st = upload_tables(c);
    if (st != LPM_OK) return st;
    if (!c->tiles_valid) {
        st = build_tiles(c);
        if (st != LPM_OK) return st;
    }
    StepParams P;
    fill_params(c, P);
    const bool batched = g.n_scenarios > 1;
    const int T = c->block * c->ppt;
    const long long E = c->sort_every, Et = c->tiles_E;
    const long long k_end = c->k + n;

    // ---- plan: segments end at snapshot steps and at multiples of E (sort points) ----------
    std::vector<Segment> plan;
    size_t keys_need = 0;
    long long upto = c->sorted_upto;
    for (long long k = c->k; k < k_end;) {
        Segment sg{};
        const long long next_bin = (k / g.bin_every + 1) * (long long)g.bin_every;
        long long e = std::min(k_end, std::min(next_bin, (long long)g.n_steps));
        if (E > 0) e = std::min(e, (k / E + 1) * E);
        sg.k = k;
        sg.e = e;
        sg.do_bin = (e % g.bin_every == 0) || e == g.n_steps;
        if (E > 0 && k > 0 && k % E == 0 && upto < k) {
            sg.sort = true;
            sg.sort_has_a = upto > 0;
            sg.sort_a_bound = upto > 0 ? released_total(c, upto) : 0;
            sg.sort_b_lo = c->int_lo[(size_t)(upto / Et)];
            sg.sort_b_hi = c->int_lo[(size_t)(k / Et)];
            keys_need = std::max(keys_need, (size_t)(sg.sort_a_bound +
                                                     (long long)(sg.sort_b_hi - sg.sort_b_lo) * T));
            upto = k;
        }
        sg.a_bound = upto > 0 ? released_total(c, upto) : 0;
        sg.b_lo = c->int_lo[(size_t)(upto / Et)];
        sg.b_hi = std::max(sg.b_lo, tiles_before(c, e));
        plan.push_back(sg);
        k = e;
    }
    if (upto > 0) {
        st = ensure_sort_buffers(c, std::max<size_t>(keys_need, 1));
        if (st != LPM_OK) return st;
    }

    // ---- run ------------------------------------------------------------------------------
    if (!batched) {
        long long kernels = 0;
        const bool ext_opts = P.dose_every > 0 || P.blpair != nullptr || P.n_species > 1 ||
                              P.langevin;
        const int occ_blocks = std::max(1, advance_occupancy(
            c->block, c->ppt, c->occ, false, ext_opts ? 1 : P.n_modes > 0 ? 2 : 0,
            adv_dyn_smem(P.n_lut)));
        st = run_segments(c, P, plan, c->stream, c->sorted_upto, c->cur, kernels, true,
                          occ_blocks);
        c->n_launches += kernels;
        if (st != LPM_OK) return st;
    } else {
        // the whole call as one graph, captured once per (steps, starting sort state) on a
        // private stream (the caller's may be the legacy stream, which cannot be captured)
        // and launched on the caller's stream
        lpm_ctx::Graph *gr = nullptr;
        for (auto &x : c->graphs)
            if (x.k0 == c->k && x.k1 == k_end && x.upto0 == c->sorted_upto && x.cur0 == c->cur)
                gr = &x;
        if (!gr) {
            if (!c->cap_stream)
                LPM_CUDA(c, cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
            const cudaStream_t cs = c->cap_stream;
            const bool ext_opts = P.dose_every > 0 || P.blpair != nullptr || P.n_species > 1 ||
                                  P.langevin;
            const int occ_blocks = std::max(1, advance_occupancy(
                c->block, c->ppt, c->occ, true, ext_opts ? 1 : P.n_modes > 0 ? 2 : 0,
                adv_dyn_smem(P.n_lut)));
            lpm_ctx::Graph ng{};
            ng.k0 = c->k;
            ng.k1 = k_end;
            ng.upto0 = ng.upto1 = c->sorted_upto;
            ng.cur0 = ng.cur1 = c->cur;
            LPM_CUDA(c, cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
            lpm_status rs = run_segments(c, P, plan, cs, ng.upto1, ng.cur1, ng.kernels, false,
                                         occ_blocks);
            cudaGraph_t graph = nullptr;
            const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
            if (rs != LPM_OK || ce != cudaSuccess) {
                if (graph) cudaGraphDestroy(graph);
                (void)cudaGetLastError();
                if (rs != LPM_OK) return rs;
                return fail(c, LPM_E_CUDA, "capturing the batched step failed: %s",
                            cudaGetErrorString(ce));
            }
            const cudaError_t ie = cudaGraphInstantiate(&ng.exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ie != cudaSuccess) {
                (void)cudaGetLastError();
                return fail(c, LPM_E_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
            }
            c->graphs.push_back(ng);
            gr = &c->graphs.back();
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        if (c->profiling) {
            e0 = next_event(c);
            e1 = next_event(c);
            if (!e0 || !e1) return fail(c, LPM_E_CUDA, "cudaEventCreate failed");
            LPM_CUDA(c, cudaEventRecord(e0, c->stream));
        }
        LPM_CUDA(c, cudaGraphLaunch(gr->exec, c->stream));
        c->slot_map_stale = true;                // (when the graph holds sorts)
        if (e1) LPM_CUDA(c, cudaEventRecord(e1, c->stream));
        c->n_launches += gr->kernels;
        c->n_adv_launches++;
        c->sorted_upto = gr->upto1;
        c->cur = gr->cur1;
    }
    for (const Segment &sg : plan)
        if (sg.do_bin) c->n_bins++;
    if (P.dose_every > 0) c->n_dose += k_end / P.dose_every - c->k / P.dose_every;
    c->k = k_end;
    return LPM_OK;
}

lpm_status lpm_current_step(const lpm_ctx *c, int64_t *k)
{
    if (!c || !k) return LPM_E_INVALID;
    *k = c->k;
    return LPM_OK;
}

lpm_status lpm_sync(lpm_ctx *c)
{
    if (!c) return LPM_E_INVALID;
    return check_device_error(c);
}

namespace {
// Converts n 64-bit fixed-point sums to doubles (x f) on the device and copies them to the
// host; the conversion and the copy run on the context stream, then it is synchronised.
lpm_status read_fixed(lpm_ctx *c, const unsigned long long *src, size_t n, double f, double *out)
{
    if (n > c->d_conv_cap) {
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        if (c->d_conv) cudaFree(c->d_conv);
        c->d_conv = nullptr;
        c->d_conv_cap = 0;
        LPM_CUDA(c, cudaMalloc(&c->d_conv, n * sizeof(double)));
        c->d_conv_cap = n;
    }
    LPM_CUDA(c, launch_fixed_to_double(c->stream, src, c->d_conv, (long long)n, f));
    c->n_launches++;
    LPM_CUDA(c, cudaMemcpyAsync(out, c->d_conv, n * sizeof(double), cudaMemcpyDeviceToHost,
                                c->stream));
    LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LPM_OK;
}
}  // namespace

lpm_status lpm_concentration(lpm_ctx *c, int scenario, double *out, size_t n_out)
{
    if (!c) return LPM_E_INVALID;
    if (scenario < 0 || scenario >= c->cfg.n_scenarios) return fail(c, LPM_E_INVALID, "bad scenario");
    if (!out || n_out != c->ncell())
        return fail(c, LPM_E_INVALID, "out must hold cz*cy*cx = %zu doubles", c->ncell());
    lpm_status st = check_device_error(c);
    if (st != LPM_OK) return st;
    const lpm_config &g = c->cfg;
    const double f = std::ldexp(1.0, -c->scen[(size_t)scenario].shift) / (g.cdx * g.cdy * g.cdz);
    return read_fixed(c, c->d_conc + (size_t)scenario * c->ncell(), c->ncell(), f, out);
}

lpm_status lpm_deposition(lpm_ctx *c, int scenario, double *dry, double *wet, size_t n_out)
{
    if (!c) return LPM_E_INVALID;
    if (scenario < 0 || scenario >= c->cfg.n_scenarios) return fail(c, LPM_E_INVALID, "bad scenario");
    const size_t plane = (size_t)c->cfg.cx * c->cfg.cy;
    if (n_out != plane) return fail(c, LPM_E_INVALID, "n_out must be cy*cx = %zu", plane);
    lpm_status st = check_device_error(c);
    if (st != LPM_OK) return st;
    const double f = std::ldexp(1.0, -c->scen[(size_t)scenario].shift) / (c->cfg.cdx * c->cfg.cdy);
    const unsigned long long *src = c->d_dep + (size_t)scenario * c->ndep();
    if (dry && (st = read_fixed(c, src, plane, f, dry)) != LPM_OK) return st;
    if (wet && (st = read_fixed(c, src + plane, plane, f, wet)) != LPM_OK) return st;
    return LPM_OK;
}

lpm_status lpm_budget(lpm_ctx *c, int scenario, double out[8])
{
    if (!c || !out) return LPM_E_INVALID;
    if (scenario < 0 || scenario >= c->cfg.n_scenarios) return fail(c, LPM_E_INVALID, "bad scenario");
    const ScenHost &h = c->scen[(size_t)scenario];
    if (!h.released) return fail(c, LPM_E_STATE, "scenario %d not released", scenario);
    lpm_status st = upload_tables(c);
    if (st != LPM_OK) return st;
    const size_t ns = (size_t)c->cfg.n_scenarios;
    for (int i : {(int)C_AIR_IN, (int)C_AIR_OUT, (int)C_N_ACTIVE})
        LPM_CUDA(c, cudaMemsetAsync(c->d_ctr + i * ns, 0, ns * sizeof(unsigned long long),
                                    c->stream));
    StepParams P;
    fill_params(c, P);
    const bool sorted = c->sorted_upto > 0;
    {
        const lpm_status sm = ensure_slot_map(c);
        if (sm != LPM_OK) return sm;
    }
    LPM_CUDA(c, launch_budget(c->stream, P, c->d_state, c->n_slots_used, c->d_slot_of,
                              c->d_sorted[c->cur], c->d_pidx[c->cur], sorted ? c->d_live : nullptr,
                              sorted ? released_total(c, c->sorted_upto) : 0, (int)c->k));
    c->n_launches++;
    st = check_device_error(c);
    if (st != LPM_OK) return st;
    unsigned long long v[N_COUNTERS];
    st = read_counters(c, scenario, v);
    if (st != LPM_OK) return st;
    const double f = std::ldexp(1.0, -h.shift);
    // initial mass of the held particles released before the current step
    double released = 0.0;
    const long long S = h.rel_last - h.rel_first;
    for (long long s = h.rel_first; s < std::min<long long>(h.rel_last, c->k); ++s) {
        const long long j = s - h.rel_first;
        const long long a = std::max(h.part_first, (j * h.n_total + S - 1) / S);
        const long long b = std::min(h.part_first + h.n, ((j + 1) * h.n_total + S - 1) / S);
        if (b > a) released += (double)(b - a) * h.m0[(size_t)j];
    }
    out[LPM_B_RELEASED] = released;
    out[LPM_B_AIR_IN] = (double)v[C_AIR_IN] * f;
    out[LPM_B_AIR_OUT] = (double)v[C_AIR_OUT] * f;
    out[LPM_B_DRY] = (double)v[C_DEP_DRY] * f;
    out[LPM_B_WET] = (double)v[C_DEP_WET] * f;
    out[LPM_B_EXITED] = (double)v[C_EXITED] * f;
    out[LPM_B_DECAYED] = released - (out[1] + out[2] + out[3] + out[4] + out[5]);
    out[LPM_B_N_ACTIVE] = (double)v[C_N_ACTIVE];
    return LPM_OK;
}

lpm_status lpm_particles(lpm_ctx *c, int64_t first, int64_t count, float *xyz, uint32_t *tag)
{
    if (!c) return LPM_E_INVALID;
    if (first < 0 || count < 0 || first + count > c->n_slots_used)
        return fail(c, LPM_E_INVALID, "slots [%lld, %lld) outside the %lld released",
                    (long long)first, (long long)(first + count), c->n_slots_used);
    lpm_status st = check_device_error(c);
    if (st != LPM_OK) return st;
    if (count == 0) return LPM_OK;
    std::vector<float4> h((size_t)count);
    if (c->d_sorted[0]) {
        // slot order: gather from the home slots, the sorted set and the dead array into
        // the spare sorted buffer (free until the next sort)
        float4 *tmp = c->d_sorted[1 - c->cur];
        {
            const lpm_status sm = ensure_slot_map(c);
            if (sm != LPM_OK) return sm;
        }
        LPM_CUDA(c, launch_gather(c->stream, c->d_state, c->d_sorted[c->cur], c->d_slot_of,
                                  c->d_grave, first, count, tmp));
        LPM_CUDA(c, cudaMemcpyAsync(h.data(), tmp, h.size() * sizeof(float4),
                                    cudaMemcpyDeviceToHost, c->stream));
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        c->n_launches++;
    } else {
        LPM_CUDA(c, cudaMemcpy(h.data(), c->d_state + first, h.size() * sizeof(float4),
                               cudaMemcpyDeviceToHost));
    }
    for (size_t i = 0; i < h.size(); ++i) {
        if (xyz) {
            xyz[3 * i] = h[i].x;
            xyz[3 * i + 1] = h[i].y;
            xyz[3 * i + 2] = h[i].z;
        }
        if (tag) {
            uint32_t t;
            std::memcpy(&t, &h[i].w, sizeof t);
            tag[i] = t;
        }
    }
    return LPM_OK;
}

lpm_status lpm_fixed_state(lpm_ctx *c, int scenario, uint64_t *conc, size_t n_conc, uint64_t *dep,
                           size_t n_dep, int64_t counters[16], int *shift)
{
    if (!c) return LPM_E_INVALID;
    if (scenario < 0 || scenario >= c->cfg.n_scenarios) return fail(c, LPM_E_INVALID, "bad scenario");
    if (conc && n_conc != c->ncell()) return fail(c, LPM_E_INVALID, "n_conc must be %zu", c->ncell());
    if (dep && n_dep != c->ndep()) return fail(c, LPM_E_INVALID, "n_dep must be %zu", c->ndep());
    lpm_status st = check_device_error(c);
    if (st != LPM_OK) return st;
    if (conc)
        LPM_CUDA(c, cudaMemcpy(conc, c->d_conc + (size_t)scenario * c->ncell(),
                               n_conc * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (dep)
        LPM_CUDA(c, cudaMemcpy(dep, c->d_dep + (size_t)scenario * c->ndep(),
                               n_dep * sizeof(uint64_t), cudaMemcpyDeviceToHost));
    if (counters) {
        unsigned long long v[N_COUNTERS];
        st = read_counters(c, scenario, v);
        if (st != LPM_OK) return st;
        for (int i = 0; i < 16; ++i) counters[i] = (int64_t)v[i];
        counters[C_N_BINS] = c->n_bins;
    }
    if (shift) *shift = c->scen[(size_t)scenario].shift;
    return LPM_OK;
}

lpm_status lpm_device_state(lpm_ctx *c, int scenario, const uint64_t **conc, const uint64_t **dep,
                            const uint64_t **counters, int64_t *counter_stride)
{
    if (!c) return LPM_E_INVALID;
    if (scenario < 0 || scenario >= c->cfg.n_scenarios) return fail(c, LPM_E_INVALID, "bad scenario");
    const size_t s = (size_t)scenario;
    if (conc) *conc = reinterpret_cast<const uint64_t *>(c->d_conc + s * c->ncell());
    if (dep) *dep = reinterpret_cast<const uint64_t *>(c->d_dep + s * c->ndep());
    if (counters) *counters = reinterpret_cast<const uint64_t *>(c->d_ctr + s);
    if (counter_stride) *counter_stride = c->cfg.n_scenarios;
    return LPM_OK;
}

lpm_status lpm_set_sort(lpm_ctx *c, int every_steps)
{
    if (!c) return LPM_E_INVALID;
    if (every_steps < 0) return fail(c, LPM_E_INVALID, "every_steps must be >= 0");
    if (every_steps == c->sort_every) return LPM_OK;
    // the sort points move: every particle returns home, the next sort starts afresh
    lpm_status st = clear_sort_state(c, true);
    if (st != LPM_OK) return st;
    c->sort_every = every_steps;
    c->tiles_valid = false;
    drop_graphs(c);
    return LPM_OK;
}

lpm_status lpm_set_langevin(lpm_ctx *c, int on, double t_lagr)
{
    if (!c) return LPM_E_INVALID;
    if (c->k != 0) return fail(c, LPM_E_STATE, "choose the Langevin variant before stepping (or after lpm_reset)");
    if (on && (!is_finite(t_lagr) || !(t_lagr > 0)))
        return fail(c, LPM_E_INVALID, "the Lagrangian time scale must be > 0");
    if (on && (!c->d_w_home || !c->d_w_sorted[0] || !c->d_w_sorted[1])) {
        const size_t n = (size_t)c->cfg.max_particles;
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        if (!c->d_w_home) {
            LPM_CUDA(c, cudaMalloc(&c->d_w_home, n * sizeof(float)));
            LPM_CUDA(c, cudaMemsetAsync(c->d_w_home, 0, n * sizeof(float), c->stream));
        }
        for (int b = 0; b < 2; ++b)
            if (!c->d_w_sorted[b]) LPM_CUDA(c, cudaMalloc(&c->d_w_sorted[b], n * sizeof(float)));
    }
    c->langevin = on ? 1 : 0;
    if (on) c->t_lagr = t_lagr;
    drop_graphs(c);                          // the graphs hold the step parameters
    return LPM_OK;
}

lpm_status lpm_particle_velocity(lpm_ctx *c, int64_t first, int64_t count, float *w)
{
    if (!c || !w) return LPM_E_INVALID;
    if (!c->langevin) return fail(c, LPM_E_STATE, "the Langevin variant is off");
    if (first < 0 || count < 0 || first + count > c->n_slots_used)
        return fail(c, LPM_E_INVALID, "slots [%lld, %lld) outside the %lld released",
                    (long long)first, (long long)(first + count), c->n_slots_used);
    lpm_status st = check_device_error(c);
    if (st != LPM_OK) return st;
    if (count == 0) return LPM_OK;
    float *tmp = c->d_w_sorted[1 - c->cur];  // free until the next sort
    {
        const lpm_status sm = ensure_slot_map(c);
        if (sm != LPM_OK) return sm;
    }
    LPM_CUDA(c, launch_gather_w(c->stream, c->d_w_home, c->d_w_sorted[c->cur], c->d_slot_of,
                                first, count, tmp));
    LPM_CUDA(c, cudaMemcpyAsync(w, tmp, (size_t)count * sizeof(float), cudaMemcpyDeviceToHost,
                                c->stream));
    LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->n_launches++;
    return LPM_OK;
}

lpm_status lpm_set_decay_chain(lpm_ctx *c, int n_species, const double *half_lives)
{
    if (!c) return LPM_E_INVALID;
    if (c->k != 0) return fail(c, LPM_E_STATE, "set the decay chain before stepping (or after lpm_reset)");
    if (n_species < 1 || n_species > MAX_SPECIES || (n_species > 1 && !half_lives))
        return fail(c, LPM_E_INVALID, "a chain has 1 to %d species", MAX_SPECIES);
    const lpm_config &g = c->cfg;
    double lam[MAX_SPECIES] = {};
    if (n_species > 1) {
        if (!is_finite(half_lives[0]) ||
            std::fabs(half_lives[0] - g.half_life_s) > 1e-9 * std::fabs(g.half_life_s) ||
            !(half_lives[0] > 0))
            return fail(c, LPM_E_INVALID, "the first half-life must be the configured one (%g s)",
                        g.half_life_s);
        for (int j = 0; j < n_species; ++j) {
            if (!is_finite(half_lives[j]) || half_lives[j] < 0 ||
                (half_lives[j] == 0 && j != n_species - 1))
                return fail(c, LPM_E_INVALID, "half-lives must be > 0 (0 = stable, last only)");
            lam[j] = half_lives[j] > 0 ? std::log(2.0) / half_lives[j] : 0.0;
            for (int i = 0; i < j; ++i)
                if (std::fabs(lam[j] - lam[i]) <= 1e-9 * std::max(lam[j], lam[i]))
                    return fail(c, LPM_E_INVALID, "decay rates of a chain must be distinct");
        }
    }
    // closed-form amounts of the rate equations: c[j][i] = prod_{k<j} l_k / prod_{k<=j,k!=i} (l_k - l_i)
    std::memset(c->chain_c, 0, sizeof c->chain_c);
    std::memset(c->chain_l, 0, sizeof c->chain_l);
    for (int j = 0; j < n_species && n_species > 1; ++j) {
        double pre = 1.0;
        for (int k = 0; k < j; ++k) pre *= lam[k];
        for (int i = 0; i <= j; ++i) {
            double den = 1.0;
            for (int k = 0; k <= j; ++k)
                if (k != i) den *= lam[k] - lam[i];
            c->chain_c[j][i] = pre / den;
        }
        c->chain_l[j] = lam[j];
    }
    const size_t ns = (size_t)g.n_scenarios;
    LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    for (unsigned long long **p : {&c->d_sp_conc, &c->d_sp_dep})
        if (*p) {
            cudaFree(*p);
            *p = nullptr;
        }
    c->n_species = 1;
    if (n_species > 1) {
        const size_t nd = (size_t)(n_species - 1) * ns;
        LPM_CUDA(c, cudaMalloc(&c->d_sp_conc, nd * c->ncell() * 8));
        LPM_CUDA(c, cudaMalloc(&c->d_sp_dep, nd * c->ndep() * 8));
        LPM_CUDA(c, cudaMemsetAsync(c->d_sp_conc, 0, nd * c->ncell() * 8, c->stream));
        LPM_CUDA(c, cudaMemsetAsync(c->d_sp_dep, 0, nd * c->ndep() * 8, c->stream));
    }
    c->n_species = n_species;
    drop_graphs(c);                          // the graphs hold the step parameters
    return LPM_OK;
}

lpm_status lpm_species(lpm_ctx *c, int scenario, int species, double *conc, double *dry,
                       double *wet, uint64_t *conc_fixed, uint64_t *dep_fixed)
{
    if (!c) return LPM_E_INVALID;
    if (scenario < 0 || scenario >= c->cfg.n_scenarios) return fail(c, LPM_E_INVALID, "bad scenario");
    if (species < 0 || species >= c->n_species)
        return fail(c, LPM_E_INVALID, "species %d outside the chain of %d", species, c->n_species);
    lpm_status st = check_device_error(c);
    if (st != LPM_OK) return st;
    const size_t ns = (size_t)c->cfg.n_scenarios, plane = (size_t)c->cfg.cx * c->cfg.cy;
    const unsigned long long *dc, *dd;
    if (species == 0) {
        dc = c->d_conc + (size_t)scenario * c->ncell();
        dd = c->d_dep + (size_t)scenario * c->ndep();
    } else {
        dc = c->d_sp_conc + ((size_t)(species - 1) * ns + scenario) * c->ncell();
        dd = c->d_sp_dep + ((size_t)(species - 1) * ns + scenario) * c->ndep();
    }
    std::vector<unsigned long long> hc(c->ncell()), hd(c->ndep());
    LPM_CUDA(c, cudaMemcpy(hc.data(), dc, hc.size() * 8, cudaMemcpyDeviceToHost));
    LPM_CUDA(c, cudaMemcpy(hd.data(), dd, hd.size() * 8, cudaMemcpyDeviceToHost));
    if (conc_fixed) std::memcpy(conc_fixed, hc.data(), hc.size() * 8);
    if (dep_fixed) std::memcpy(dep_fixed, hd.data(), hd.size() * 8);
    const lpm_config &g = c->cfg;
    const double unit = std::ldexp(1.0, -c->scen[(size_t)scenario].shift);
    if (conc)
        for (size_t i = 0; i < hc.size(); ++i) conc[i] = (double)hc[i] * unit / (g.cdx * g.cdy * g.cdz);
    for (int kind = 0; kind < 2; ++kind) {
        double *out = kind ? wet : dry;
        if (!out) continue;
        for (size_t i = 0; i < plane; ++i)
            out[i] = (double)hd[kind * plane + i] * unit / (g.cdx * g.cdy);
    }
    return LPM_OK;
}

lpm_status lpm_set_kz_model(lpm_ctx *c, int model, double kz_min)
{
    if (!c) return LPM_E_INVALID;
    if (model < 0 || model > 1) return fail(c, LPM_E_INVALID, "K_z model must be 0 or 1");
    if (!is_finite(kz_min) || kz_min < 0) return fail(c, LPM_E_INVALID, "kz_min must be >= 0");
    const lpm_config &g = c->cfg;
    if (model == 1 && (!c->d_bl || !c->d_blpair)) {
        const size_t cols = (size_t)g.nx * g.ny;
        const size_t n_pair = (size_t)std::max(1, g.n_met_t - 1);
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        if (!c->d_bl) LPM_CUDA(c, cudaMalloc(&c->d_bl, cols * g.n_met_t * sizeof(float4)));
        if (!c->d_blpair)
            LPM_CUDA(c, cudaMalloc(&c->d_blpair, cols * n_pair * 2 * sizeof(float4)));
        c->bl_set.assign((size_t)g.n_met_t, 0);
    }
    c->kz_model = model;
    c->kz_min = kz_min;
    drop_graphs(c);                          // the graphs hold the step parameters
    return LPM_OK;
}

lpm_status lpm_set_boundary_layer(lpm_ctx *c, int t_index, const float *bl, int on_device)
{
    if (!c) return LPM_E_INVALID;
    const lpm_config &g = c->cfg;
    if (!c->d_bl || !c->d_blpair || c->bl_set.empty())
        return fail(c, LPM_E_STATE, "select K_z model 1 (lpm_set_kz_model) first");
    if (t_index < 0 || t_index >= g.n_met_t)
        return fail(c, LPM_E_INVALID, "t_index %d outside [0, %d)", t_index, g.n_met_t);
    if (!bl) return fail(c, LPM_E_INVALID, "bl is NULL");
    const size_t cols = (size_t)g.nx * g.ny;
    if (!on_device) {
        for (size_t i = 0; i < cols; ++i) {
            const float *v = bl + 4 * i;
            if (!std::isfinite(v[0]) || !std::isfinite(v[1]) || !std::isfinite(v[2]) ||
                v[0] < 0.0f || !(v[2] > 0.0f))
                return fail(c, LPM_E_INVALID, "column %zu: need u* >= 0, finite 1/L, H_z > 0", i);
        }
    }
    LPM_CUDA(c, cudaMemcpyAsync(c->d_bl + cols * t_index, bl, cols * sizeof(float4),
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                c->stream));
    c->bl_set[(size_t)t_index] = 1;
    // time pairs (h, h+1) that this slab completes
    for (int h = t_index - 1; h <= t_index; ++h) {
        const int h1 = g.n_met_t > 1 ? h + 1 : h;
        if (h < 0 || h1 > g.n_met_t - 1 || (g.n_met_t > 1 && h > g.n_met_t - 2)) continue;
        if (!c->bl_set[(size_t)h] || !c->bl_set[(size_t)h1]) continue;
        LPM_CUDA(c, launch_pack(c->stream, c->d_bl + cols * h, c->d_bl + cols * h1, nullptr,
                                nullptr, c->d_blpair + cols * 2 * h, nullptr, g.nx, g.ny, 1));
        c->n_launches++;
    }
    if (!on_device) LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    return LPM_OK;
}

lpm_status lpm_set_dosage(lpm_ctx *c, int every_steps)
{
    if (!c) return LPM_E_INVALID;
    if (every_steps < 0) return fail(c, LPM_E_INVALID, "every_steps must be >= 0");
    const size_t ns = (size_t)c->cfg.n_scenarios;
    if (every_steps > 0 && !c->d_dose) {
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        LPM_CUDA(c, cudaMalloc(&c->d_dose, ns * c->ncell() * sizeof(unsigned long long)));
    }
    if (c->d_dose)
        LPM_CUDA(c, cudaMemsetAsync(c->d_dose, 0, ns * c->ncell() * sizeof(unsigned long long),
                                    c->stream));
    LPM_CUDA(c, cudaMemsetAsync(c->d_ctr + (size_t)C_DOSE_OUT * ns, 0,
                                ns * sizeof(unsigned long long), c->stream));
    c->dose_every = every_steps;
    c->dose_bits = 0;
    if (every_steps > 0) {
        // up to floor(S / n) samples of at most the total mass: b bits fewer than the
        // snapshots keep every sum below 2^61 units
        const long long most = c->cfg.n_steps / every_steps;
        while (c->dose_bits < 62 && (1LL << c->dose_bits) < most) ++c->dose_bits;
    }
    c->n_dose = 0;
    drop_graphs(c);                          // the graphs hold the step parameters
    return LPM_OK;
}

lpm_status lpm_dosage(lpm_ctx *c, int scenario, double *out, size_t n_out, uint64_t *fixed,
                      int64_t *n_samples)
{
    if (!c) return LPM_E_INVALID;
    if (scenario < 0 || scenario >= c->cfg.n_scenarios) return fail(c, LPM_E_INVALID, "bad scenario");
    if (!c->d_dose) return fail(c, LPM_E_STATE, "dosage was never enabled (lpm_set_dosage)");
    if ((out || fixed) && n_out != c->ncell())
        return fail(c, LPM_E_INVALID, "n_out must be cz*cy*cx = %zu", c->ncell());
    lpm_status st = check_device_error(c);
    if (st != LPM_OK) return st;
    if (n_samples) *n_samples = c->n_dose;
    if (!out && !fixed) return LPM_OK;
    std::vector<unsigned long long> h(c->ncell());
    LPM_CUDA(c, cudaMemcpy(h.data(), c->d_dose + (size_t)scenario * c->ncell(),
                           h.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    if (fixed) std::memcpy(fixed, h.data(), h.size() * sizeof(uint64_t));
    if (out) {
        const lpm_config &g = c->cfg;
        const double f = std::ldexp(1.0, c->dose_bits - c->scen[(size_t)scenario].shift) *
                         ((double)c->dose_every * g.dt) / (g.cdx * g.cdy * g.cdz);
        for (size_t i = 0; i < h.size(); ++i) out[i] = (double)h[i] * f;
    }
    return LPM_OK;
}

lpm_status lpm_set_params(lpm_ctx *c, double k_scale, double bias_u, double bias_v)
{
    if (!c) return LPM_E_INVALID;
    if (!(k_scale > 0) || !is_finite(k_scale) || !is_finite(bias_u) || !is_finite(bias_v))
        return fail(c, LPM_E_INVALID, "k_scale must be > 0 and the bias finite");
    if (c->k_scale == k_scale && c->bias_u == bias_u && c->bias_v == bias_v) return LPM_OK;
    c->k_scale = k_scale;
    c->bias_u = bias_u;
    c->bias_v = bias_v;
    c->params_version++;
    drop_graphs(c);
    return LPM_OK;
}

lpm_status lpm_set_emission(lpm_ctx *c, int scenario, const double *q, int n_q)
{
    if (!c) return LPM_E_INVALID;
    if (scenario < 0 || scenario >= c->n_released)
        return fail(c, LPM_E_STATE, "scenario %d has not been released", scenario);
    if (c->k != 0) return fail(c, LPM_E_STATE, "emission can change only at step 0 (after lpm_reset)");
    if (!q || n_q < 1 || n_q > MAX_NQ) return fail(c, LPM_E_INVALID, "need 1 <= n_q <= %d", MAX_NQ);
    for (int i = 0; i < n_q; ++i)
        if (!is_finite(q[i]) || q[i] < 0) return fail(c, LPM_E_INVALID, "emission rates must be >= 0");
    ScenHost &h = c->scen[(size_t)scenario];
    if (h.q.size() == (size_t)n_q && std::equal(h.q.begin(), h.q.end(), q)) return LPM_OK;
    h.q.assign(q, q + n_q);
    lpm_status st = assign_masses(c, h);
    if (st != LPM_OK) return st;
    c->tables_dirty = true;
    return LPM_OK;
}

namespace {

int adj_nq(const lpm_ctx *c)
{
    size_t nq = 1;
    for (const ScenHost &h : c->scen) nq = std::max(nq, h.q.size());
    return (int)nq;
}

// Segments of the sorted form: segment s covers steps [s CK, (s+1) CK); its entries are
// blocks over the particles of every scenario released before s CK (a bound of those
// alive) and the tiles, scenario by scenario, of the particles released within it; its
// trajectory rows and end states are laid out back to back.
lpm_status adj_plan_segments(lpm_ctx *c)
{
    lpm_ctx::AdjSorted &S = c->as;
    const long long NS = c->cfg.n_steps;
    const int n_seg = (int)((NS + CK - 1) / CK);
    S.tiles.clear();
    S.seg_tile.assign((size_t)n_seg + 1, 0);
    S.tiles_a.assign((size_t)n_seg, 0);
    S.off.assign((size_t)n_seg + 1, 0);
    S.foff.assign((size_t)n_seg + 1, 0);
    S.ckoff.assign((size_t)n_seg + 1, 0);
    S.max_width = 0;
    long long off = 0, foff = 0, ckoff = 0;
    for (int s = 0; s < n_seg; ++s) {
        S.seg_tile[(size_t)s] = (int)S.tiles.size();
        long long a = 0;
        for (size_t q = 0; q < c->scen.size(); ++q) {
            const ScenHost &h = c->scen[q];
            const long long a_q = released_before(h, (long long)s * CK);
            const long long b_q = released_before(h, (long long)(s + 1) * CK);
            a += a_q;
            for (long long p = a_q; p < b_q; p += ADJ_BLOCK) {
                Tile t;
                t.scen = (int)q;
                t.first = h.first_slot + p;
                t.count = (int)std::min<long long>(ADJ_BLOCK, b_q - p);
                S.tiles.push_back(t);
            }
        }
        S.tiles_a[(size_t)s] = s ? (int)((a + ADJ_BLOCK - 1) / ADJ_BLOCK) : 0;
        const long long width =
            (long long)(S.tiles_a[(size_t)s] + (int)S.tiles.size() - S.seg_tile[(size_t)s]) * ADJ_BLOCK;
        S.off[(size_t)s] = off;
        S.foff[(size_t)s] = foff;
        S.ckoff[(size_t)s] = ckoff;
        off += std::min<long long>(CK, NS - (long long)s * CK) * width;
        foff += width;
        ckoff += (long long)S.tiles_a[(size_t)s] * ADJ_BLOCK;
        S.max_width = std::max(S.max_width, width);
    }
    S.seg_tile[(size_t)n_seg] = (int)S.tiles.size();
    S.off[(size_t)n_seg] = off;
    S.foff[(size_t)n_seg] = foff;
    S.ckoff[(size_t)n_seg] = ckoff;
    LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    if (S.d_tiles) cudaFree(S.d_tiles);
    S.d_tiles = nullptr;
    LPM_CUDA(c, cudaMalloc(&S.d_tiles, std::max<size_t>(1, S.tiles.size()) * sizeof(Tile)));
    if (!S.tiles.empty())
        LPM_CUDA(c, cudaMemcpy(S.d_tiles, S.tiles.data(), S.tiles.size() * sizeof(Tile),
                               cudaMemcpyHostToDevice));
    return LPM_OK;
}

// Sort keys of the adjoint's segments: cells for one scenario; with several, scenario and
// cell tile, so that each scenario's particles stay together (blocks of one scenario keep
// their receptor sums and gradients in shared memory).
int adj_key_scen(const lpm_ctx *c)
{
    return c->scen.size() > 1 ? (int)c->scen.size() : 0;
}

// The sorted form's own buffers (allocates whatever is still missing).
lpm_status adj_sorted_buffers(lpm_ctx *c)
{
    lpm_ctx::AdjSorted &S = c->as;
    const size_t ns = std::max<size_t>(1, (size_t)c->n_slots_used);
    const size_t nseg = S.tiles_a.size();
    const size_t nb = (size_t)sort_dead_key(c->cfg.nx, c->cfg.ny, c->cfg.nz, adj_key_scen(c)) + 1;
    auto need = [&](auto *&p, size_t bytes) -> cudaError_t {
        return p ? cudaSuccess : cudaMalloc(&p, bytes);
    };
    LPM_CUDA(c, need(S.ord, std::max<size_t>(1, nseg) * ns * sizeof(unsigned int)));
    LPM_CUDA(c, need(S.live, std::max<size_t>(1, nseg) * sizeof(unsigned int)));
    LPM_CUDA(c, need(S.keys, (size_t)std::max<long long>(1, S.max_width) * sizeof(unsigned int)));
    LPM_CUDA(c, need(S.hist, nb * sizeof(unsigned int)));
    LPM_CUDA(c, need(S.bsums, ((nb + 1023) / 1024) * sizeof(unsigned int)));
    LPM_CUDA(c, need(S.meta, 4 * sizeof(unsigned int)));
    LPM_CUDA(c, need(S.grave_n, sizeof(unsigned int)));
    for (float4 **p : {&S.st[0], &S.st[1], &S.home, &S.mu, &S.grave})
        LPM_CUDA(c, need(*p, ns * sizeof(float4)));
    return LPM_OK;
}

// Segment s of the sorted form, its sorted entries in S.st[cur]. Trajectory form: its rows
// and end states within the whole trajectory; checkpoint form: its checkpoint, and the
// scratch for its rows and end states.
AdjSeg adj_segment(const lpm_ctx *c, int s, int cur)
{
    const lpm_ctx::AdjSorted &S = c->as;
    AdjSeg G;
    G.k_lo = s * CK;
    G.k_hi = (int)std::min<long long>(c->cfg.n_steps, (long long)(s + 1) * CK);
    G.live = S.live + s;
    G.ord = S.ord + (size_t)s * std::max<size_t>(1, (size_t)c->n_slots_used);
    G.sorted = S.st[cur];
    G.tiles_a = S.tiles_a[(size_t)s];
    G.home = S.home;
    G.tiles = S.d_tiles;
    G.b_first = S.seg_tile[(size_t)s];
    G.width = (long long)(G.tiles_a + S.seg_tile[(size_t)s + 1] - G.b_first) * ADJ_BLOCK;
    // checkpoint form: the scratch has two halves, segment s in half s & 1
    G.traj = c->d_traj + (c->adj_traj ? S.off[(size_t)s] : (s & 1) * (long long)CK * S.max_width);
    G.fin = c->d_fin + (c->adj_traj ? S.foff[(size_t)s] : (s & 1) * S.max_width);
    G.mu = S.mu;
    G.ck = c->adj_traj ? nullptr : c->d_ckpt + S.ckoff[(size_t)s];
    return G;
}

// Forward of the sorted form: per segment the advance over its entries, then the sort of
// the survivors (and the segment's releases) by cell into the other buffer.
lpm_status adj_forward_sorted(lpm_ctx *c, const StepParams &P, const AdjParams &A)
{
    lpm_ctx::AdjSorted &S = c->as;
    const int n_seg = (int)S.tiles_a.size();
    LPM_CUDA(c, cudaMemsetAsync(S.live, 0, std::max(1, n_seg) * sizeof(unsigned int), c->stream));
    LPM_CUDA(c, cudaMemsetAsync(S.meta, 0, 4 * sizeof(unsigned int), c->stream));
    LPM_CUDA(c, cudaMemsetAsync(S.grave_n, 0, sizeof(unsigned int), c->stream));
    int cur = 0;
    for (int s = 0; s < n_seg; ++s) {
        const AdjSeg G = adj_segment(c, s, cur);
        if (s > 0)
            LPM_CUDA(c, cudaMemcpyAsync(S.live + s, S.meta, sizeof(unsigned int),
                                        cudaMemcpyDeviceToDevice, c->stream));
        LPM_CUDA(c, launch_adj_forward_seg(c->stream, P, A, G, (int)(G.width / ADJ_BLOCK),
                                           c->adj_traj ? SEG_STORE : SEG_CKPT));
        c->n_launches++;
        if (s + 1 < n_seg) {
            SortSource in;
            in.state_a = G.sorted;
            in.pidx_a = G.ord;
            in.has_a = s > 0;
            in.a_bound = (long long)G.tiles_a * ADJ_BLOCK;
            in.state_b = S.home;
            in.tiles = S.d_tiles;
            in.b_first = G.b_first;
            in.n_b = S.seg_tile[(size_t)s + 1] - G.b_first;
            in.T = ADJ_BLOCK;
            in.w_a = in.w_b = nullptr;
            in.keys_ready = false;
            in.key_scen = adj_key_scen(c);
            SortBuffers out;
            out.state_out = S.st[cur ^ 1];
            out.pidx_out = S.ord + (size_t)(s + 1) * std::max<size_t>(1, (size_t)c->n_slots_used);
            out.slot_of = nullptr;                // the adjoint reads no slot map
            out.grave_home = nullptr;
            out.keys = S.keys;
            out.hist = S.hist;
            out.block_sums = S.bsums;
            out.meta = S.meta;
            out.grave = S.grave;
            out.grave_count = S.grave_n;
            out.w_out = nullptr;
            out.cap = std::max<long long>(1, c->n_slots_used);
            out.err = c->d_err;
            LPM_CUDA(c, launch_sort(c->stream, P, in, out));
            c->n_launches += 7;
            cur ^= 1;
        }
    }
    return LPM_OK;
}

// Backward of the checkpoint form of the sorted segments, last segment first: each
// segment is recomputed from its checkpoint (the same keyed draws and FP32 arithmetic in
// the same entry order, so the same states and events as the receptor forward) into one
// half of the scratch, on the context's second stream, so that segment s - 1 is recomputed
// into the other half while segment s is swept; each sweep waits for its own
// recomputation, and the sweeps stay in order on the context stream (they hand dL/dX down
// through G.mu).
lpm_status adj_backward_ckpt(lpm_ctx *c, const StepParams &P, const AdjParams &A)
{
    const int n_seg = (int)c->as.tiles_a.size();
    if (n_seg < 1) return LPM_OK;
    if (!c->adj_stream)
        LPM_CUDA(c, cudaStreamCreateWithFlags(&c->adj_stream, cudaStreamNonBlocking));
    for (cudaEvent_t &e : c->ev_adj)
        if (!e) LPM_CUDA(c, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    cudaEvent_t *recomputed = c->ev_adj, *swept = c->ev_adj + 2;
    auto recompute = [&](int s) -> lpm_status {
        const AdjSeg G = adj_segment(c, s, 0);
        LPM_CUDA(c, launch_adj_forward_seg(c->adj_stream, P, A, G, (int)(G.width / ADJ_BLOCK),
                                           SEG_RECOMPUTE));
        LPM_CUDA(c, cudaEventRecord(recomputed[s & 1], c->adj_stream));
        c->n_launches++;
        return LPM_OK;
    };
    LPM_CUDA(c, cudaEventRecord(c->ev_adj[4], c->stream));       // the forward's states
    LPM_CUDA(c, cudaStreamWaitEvent(c->adj_stream, c->ev_adj[4], 0));
    lpm_status st = recompute(n_seg - 1);
    if (st != LPM_OK) return st;
    for (int s = n_seg - 1; s >= 0; --s) {
        if (s > 0) {
            // half (s - 1) & 1 was last read by the sweep of segment s + 1
            if (s + 1 < n_seg)
                LPM_CUDA(c, cudaStreamWaitEvent(c->adj_stream, swept[(s + 1) & 1], 0));
            if ((st = recompute(s - 1)) != LPM_OK) return st;
        }
        const AdjSeg G = adj_segment(c, s, 0);
        LPM_CUDA(c, cudaStreamWaitEvent(c->stream, recomputed[s & 1], 0));
        LPM_CUDA(c, launch_adj_backward_seg(c->stream, P, A, G, (int)(G.width / ADJ_BLOCK)));
        LPM_CUDA(c, cudaEventRecord(swept[s & 1], c->stream));
        c->n_launches++;
    }
    return LPM_OK;
}

// Backward of the sorted form, last segment first: the trajectory form sweeps the stored
// segments; the checkpoint form recomputes them (adj_backward_ckpt).
lpm_status adj_backward_sorted(lpm_ctx *c, const StepParams &P, const AdjParams &A)
{
    if (!c->adj_traj) {
        const lpm_status st = adj_backward_ckpt(c, P, A);
        // whatever ran on the second stream is ordered before the context stream's next
        // work, also when a launch failed part-way
        if (c->adj_stream && c->ev_adj[4] &&
            cudaEventRecord(c->ev_adj[4], c->adj_stream) == cudaSuccess)
            (void)cudaStreamWaitEvent(c->stream, c->ev_adj[4], 0);
        return st;
    }
    for (int s = (int)c->as.tiles_a.size() - 1; s >= 0; --s) {
        const AdjSeg G = adj_segment(c, s, 0);
        LPM_CUDA(c, launch_adj_backward_seg(c->stream, P, A, G, (int)(G.width / ADJ_BLOCK)));
        c->n_launches++;
    }
    return LPM_OK;
}

// Storage of the forward's states for the backward: the whole trajectory (nt_need rows,
// nf_need end states) when it fits in the limit and in free device memory (keeping 8 GiB
// spare), else checkpoints every CK steps. For the checkpoint form of the sorted segments
// the trajectory buffers become the recomputation's scratch (st_need rows, sf_need end states;
// `scratch` tells whether it fits in free memory); st_need = 0 frees them.
lpm_status adj_storage(lpm_ctx *c, size_t nt_need, size_t nf_need, size_t st_need,
                       size_t sf_need, bool &scratch)
{
    scratch = false;
    const size_t spare = (size_t)8 << 30;
    const size_t need_b = (nt_need + nf_need) * sizeof(float4);
    bool traj = need_b <= c->adj_store_max;
    auto free_rows = [c]() {
        for (float4 **p : {&c->d_traj, &c->d_fin}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
        c->d_traj_cap = c->d_fin_cap = 0;
        c->adj_sig.clear();
    };
    if (traj && (nt_need > c->d_traj_cap || nf_need > c->d_fin_cap)) {
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        size_t fr = 0, tot = 0;
        LPM_CUDA(c, cudaMemGetInfo(&fr, &tot));
        const size_t held = (c->d_traj_cap + c->d_fin_cap + c->d_ckpt_cap) * sizeof(float4);
        traj = need_b + spare <= fr + held;
        if (traj) {
            free_rows();
            if (c->d_ckpt) cudaFree(c->d_ckpt);
            c->d_ckpt = nullptr;
            c->d_ckpt_cap = 0;
            const size_t nt = std::max<size_t>(1, nt_need);
            const size_t nf = std::max<size_t>(1, nf_need);
            if (cudaMalloc(&c->d_traj, nt * sizeof(float4)) == cudaSuccess &&
                cudaMalloc(&c->d_fin, nf * sizeof(float4)) == cudaSuccess) {
                c->d_traj_cap = nt;
                c->d_fin_cap = nf;
            } else {
                (void)cudaGetLastError();             // out of memory: use checkpoints
                free_rows();
                traj = false;
            }
        }
    }
    if (!traj) {
        // keep buffers that hold the scratch without being more than twice its size
        const bool keep = st_need > 0 && st_need <= c->d_traj_cap && sf_need <= c->d_fin_cap &&
                          c->d_traj_cap <= 2 * st_need && c->d_fin_cap <= 2 * sf_need;
        if (keep) {
            scratch = true;
        } else {
            if (c->d_traj || c->d_fin) {
                LPM_CUDA(c, cudaStreamSynchronize(c->stream));
                free_rows();
            }
            if (st_need > 0) {
                size_t fr = 0, tot = 0;
                LPM_CUDA(c, cudaMemGetInfo(&fr, &tot));
                if ((st_need + sf_need) * sizeof(float4) + spare <= fr &&
                    cudaMalloc(&c->d_traj, st_need * sizeof(float4)) == cudaSuccess &&
                    cudaMalloc(&c->d_fin, sf_need * sizeof(float4)) == cudaSuccess) {
                    c->d_traj_cap = st_need;
                    c->d_fin_cap = sf_need;
                    scratch = true;
                } else {
                    (void)cudaGetLastError();         // no room: release-order checkpoints
                    free_rows();
                }
            }
        }
    }
    c->adj_traj = traj;
    return LPM_OK;
}

lpm_status adj_prepare(lpm_ctx *c, const double *rec, int R, double bandwidth, int every,
                       AdjParams &A, StepParams &P, bool reuse = false)
{
    const lpm_config &g = c->cfg;
    if (R < 1 || R > MAX_REC || !rec) return fail(c, LPM_E_INVALID, "need 1 <= R <= %d receptors", MAX_REC);
    if (!(bandwidth > 0) || every < 1) return fail(c, LPM_E_INVALID, "bandwidth > 0 and every >= 1");
    if (g.drift_correction) return fail(c, LPM_E_INVALID, "the adjoint does not support drift_correction");
    if (c->kz_model != 0) return fail(c, LPM_E_INVALID, "the adjoint does not support K_z from Eq. 3");
    if (c->langevin) return fail(c, LPM_E_INVALID, "the adjoint does not support the Langevin variant");
    if (c->n_modes > 0)
        return fail(c, LPM_E_INVALID, "the adjoint does not support perturbation modes");
    if (c->n_released != g.n_scenarios)
        return fail(c, LPM_E_STATE, "%d of %d scenarios released", c->n_released, g.n_scenarios);
    if (adj_nq(c) > MAX_NQ) return fail(c, LPM_E_INVALID, "emission series longer than %d", MAX_NQ);
    for (int t = 0; t < g.n_met_t; ++t)
        if (!c->met_set[(size_t)t]) return fail(c, LPM_E_STATE, "met slab %d not set", t);
    const int n_samp = (int)(g.n_steps / every);
    if (n_samp < 1) return fail(c, LPM_E_INVALID, "no sample step in the run");
    lpm_status st = upload_tables(c);
    if (st != LPM_OK) return st;
    fill_params(c, P);
    for (size_t h = 0; h < c->pair_pending.size(); ++h)      // weather still being uploaded
        if (c->pair_pending[h]) LPM_CUDA(c, cudaStreamWaitEvent(c->stream, c->ev_pair[h], 0));
    // tiles of ADJ_BLOCK particles over every held particle; the trajectory rows of a tile
    // start at its first particle's release step (release steps do not decrease with slot)
    if (!c->adj_tiles_valid) {
        c->adj_tiles.clear();
        std::vector<longlong2> tt;
        size_t rows = 0;
        for (size_t s = 0; s < c->scen.size(); ++s) {
            const ScenHost &h = c->scen[s];
            for (long long p = 0; p < h.n; p += ADJ_BLOCK) {
                Tile t;
                t.scen = (int)s;
                t.first = h.first_slot + p;
                t.count = (int)std::min<long long>(ADJ_BLOCK, h.n - p);
                c->adj_tiles.push_back(t);
                const long long k0 =
                    h.rel_first + ((h.part_first + p) * (h.rel_last - h.rel_first)) / h.n_total;
                tt.push_back(make_longlong2((long long)rows, k0));
                rows += (size_t)std::max<long long>(0, g.n_steps - k0) * ADJ_BLOCK;
            }
        }
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        for (void **p : {(void **)&c->d_adj_tiles, (void **)&c->d_traj_tile}) {
            if (*p) cudaFree(*p);
            *p = nullptr;
        }
        const size_t nt = std::max<size_t>(1, c->adj_tiles.size());
        LPM_CUDA(c, cudaMalloc(&c->d_adj_tiles, nt * sizeof(Tile)));
        LPM_CUDA(c, cudaMalloc(&c->d_traj_tile, nt * sizeof(longlong2)));
        LPM_CUDA(c, cudaMemcpy(c->d_adj_tiles, c->adj_tiles.data(), c->adj_tiles.size() * sizeof(Tile),
                               cudaMemcpyHostToDevice));
        LPM_CUDA(c, cudaMemcpy(c->d_traj_tile, tt.data(), tt.size() * sizeof(longlong2),
                               cudaMemcpyHostToDevice));
        c->traj_need = rows;
        lpm_status pst = adj_plan_segments(c);
        if (pst != LPM_OK) return pst;
        c->adj_tiles_valid = true;
    }
    if (!reuse) {
        const bool want_sorted = c->sort_every > 0;
        const lpm_ctx::AdjSorted &S = c->as;
        bool scratch = false;
        lpm_status sst =
            want_sorted ? adj_storage(c, (size_t)S.off.back(), (size_t)S.foff.back(),
                                      2 * (size_t)CK * (size_t)S.max_width,
                                      2 * (size_t)S.max_width, scratch)
                        : adj_storage(c, c->traj_need, (size_t)c->n_slots_used, 0, 0, scratch);
        if (sst != LPM_OK) return sst;
        c->adj_sorted = want_sorted && (c->adj_traj || scratch);
        if (c->adj_sorted && (sst = adj_sorted_buffers(c)) != LPM_OK) return sst;
    }
    const int n_ck = (int)((g.n_steps + CK - 1) / CK);
    // checkpoints: the sorted entries of every segment, or every slot every CK steps
    const size_t need_ck = c->adj_sorted ? (size_t)std::max<long long>(1, c->as.ckoff.back())
                                         : (size_t)n_ck * (size_t)c->n_slots_used;
    if (!c->adj_traj && need_ck > c->d_ckpt_cap) {
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        if (c->d_ckpt) cudaFree(c->d_ckpt);
        c->d_ckpt = nullptr;
        LPM_CUDA(c, cudaMalloc(&c->d_ckpt, need_ck * sizeof(float4)));
        c->d_ckpt_cap = need_ck;
    }
    const size_t ns = (size_t)g.n_scenarios;
    const int nq = adj_nq(c), ng = 3 + nq + 3;
    const size_t need_buf = std::max((size_t)MAX_REC * ns, (size_t)ng * ns);
    if (!c->d_rec) LPM_CUDA(c, cudaMalloc(&c->d_rec, MAX_REC * sizeof(float4)));
    if (need_buf > c->d_rbuf_cap) {
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        for (double *p : {c->d_rC, c->d_rw, c->d_rgrad})
            if (p) cudaFree(p);
        c->d_rC = c->d_rw = c->d_rgrad = nullptr;
        LPM_CUDA(c, cudaMalloc(&c->d_rC, need_buf * sizeof(double)));
        LPM_CUDA(c, cudaMalloc(&c->d_rw, need_buf * sizeof(double)));
        LPM_CUDA(c, cudaMalloc(&c->d_rgrad, need_buf * sizeof(double)));
        c->d_rbuf_cap = need_buf;
    }
    std::vector<float4> hr((size_t)R);
    for (int r = 0; r < R; ++r) {
        if (!is_finite(rec[3 * r]) || !is_finite(rec[3 * r + 1]) || !is_finite(rec[3 * r + 2]))
            return fail(c, LPM_E_INVALID, "receptor %d not finite", r);
        hr[(size_t)r] = make_float4((float)rec[3 * r], (float)rec[3 * r + 1], (float)rec[3 * r + 2], 0.f);
    }
    // receptor bins: the receptors' box widened by the cut-off (6 bandwidths) and a margin
    // that covers FP32 rounding of positions and bin arithmetic; bins of about the cut-off;
    // bin b lists, in increasing order, every receptor within cut-off + margin of it
    const double cut = 6.0 * bandwidth, margin = 1.0 + 1e-3 * cut;
    double rx0 = 1e300, rx1 = -1e300, ry0 = 1e300, ry1 = -1e300;
    for (const float4 &q : hr) {
        rx0 = std::min(rx0, (double)q.x); rx1 = std::max(rx1, (double)q.x);
        ry0 = std::min(ry0, (double)q.y); ry1 = std::max(ry1, (double)q.y);
    }
    const float bx0 = (float)(rx0 - cut - 2.0 * margin), by0 = (float)(ry0 - cut - 2.0 * margin);
    const double wx = rx1 + cut + 2.0 * margin - (double)bx0, wy = ry1 + cut + 2.0 * margin - (double)by0;
    double bin = cut;
    int nbx = std::max(1, (int)std::ceil(wx / bin)), nby = std::max(1, (int)std::ceil(wy / bin));
    while ((long long)nbx * nby > 4096) {
        bin *= 1.5;
        nbx = std::max(1, (int)std::ceil(wx / bin));
        nby = std::max(1, (int)std::ceil(wy / bin));
    }
    const float inv_bin = (float)(1.0 / bin);
    const double be = 1.0 / (double)inv_bin;          // the width the kernel's arithmetic uses
    nbx = std::max(1, (int)std::ceil(wx / be));
    nby = std::max(1, (int)std::ceil(wy / be));
    std::vector<int> boff((size_t)nbx * nby + 1, 0);
    std::vector<unsigned char> bidx;
    const double reach2 = (cut + margin) * (cut + margin);
    for (int by = 0; by < nby; ++by)
        for (int bxi = 0; bxi < nbx; ++bxi) {
            const double xl = (double)bx0 + bxi * be - margin, xh = (double)bx0 + (bxi + 1) * be + margin;
            const double yl = (double)by0 + by * be - margin, yh = (double)by0 + (by + 1) * be + margin;
            for (int r = 0; r < R; ++r) {
                const double qx = hr[(size_t)r].x, qy = hr[(size_t)r].y;
                const double dx = std::max(0.0, std::max(xl - qx, qx - xh));
                const double dy = std::max(0.0, std::max(yl - qy, qy - yh));
                if (dx * dx + dy * dy <= reach2) bidx.push_back((unsigned char)r);
            }
            boff[(size_t)by * nbx + bxi + 1] = (int)bidx.size();
        }
    if (boff.size() > c->d_rbin_off_cap || std::max<size_t>(1, bidx.size()) > c->d_rbin_idx_cap) {
        LPM_CUDA(c, cudaStreamSynchronize(c->stream));
        if (c->d_rbin_off) cudaFree(c->d_rbin_off);
        if (c->d_rbin_idx) cudaFree(c->d_rbin_idx);
        c->d_rbin_off = nullptr;
        c->d_rbin_idx = nullptr;
        c->d_rbin_off_cap = c->d_rbin_idx_cap = 0;
        LPM_CUDA(c, cudaMalloc(&c->d_rbin_off, boff.size() * sizeof(int)));
        LPM_CUDA(c, cudaMalloc(&c->d_rbin_idx, std::max<size_t>(1, bidx.size())));
        c->d_rbin_off_cap = boff.size();
        c->d_rbin_idx_cap = std::max<size_t>(1, bidx.size());
    }
    LPM_CUDA(c, cudaMemcpyAsync(c->d_rec, hr.data(), hr.size() * sizeof(float4),
                                cudaMemcpyHostToDevice, c->stream));
    LPM_CUDA(c, cudaMemcpyAsync(c->d_rbin_off, boff.data(), boff.size() * sizeof(int),
                                cudaMemcpyHostToDevice, c->stream));
    if (!bidx.empty())
        LPM_CUDA(c, cudaMemcpyAsync(c->d_rbin_idx, bidx.data(), bidx.size(),
                                    cudaMemcpyHostToDevice, c->stream));
    LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    std::memset(&A, 0, sizeof A);
    A.rbin_off = c->d_rbin_off;
    A.rbin_idx = c->d_rbin_idx;
    A.rbx0 = bx0;
    A.rby0 = by0;
    A.rinv_bin = inv_bin;
    A.rnbx = nbx;
    A.rnby = nby;
    const double s2 = bandwidth * bandwidth;
    A.rec = c->d_rec;
    A.R = R;
    A.inv2s2 = (float)(1.0 / (2.0 * s2));
    A.norm = (float)std::pow(2.0 * 3.14159265358979323846 * s2, -1.5);
    A.inv_s2 = (float)(1.0 / s2);
    A.cut2 = (float)(36.0 * s2);
    A.every = every;
    A.inv_ns = (float)(1.0 / n_samp);
    A.n_steps = (int)g.n_steps;
    A.n_ck = n_ck;
    A.ckpt = c->d_ckpt;
    A.n_slots = c->n_slots_used;
    A.traj = c->adj_traj ? c->d_traj : nullptr;
    A.traj_cap = (long long)c->d_traj_cap;
    A.fin = c->adj_traj ? c->d_fin : nullptr;
    A.traj_tile = c->d_traj_tile;
    A.tiles = c->d_adj_tiles;
    A.C = c->d_rC;
    A.w = c->d_rw;
    A.grad = c->d_rgrad;
    A.ng = ng;
    A.nq = nq;
    A.mq = c->d_mq;
    A.qi = c->d_qi;
    return LPM_OK;
}

std::vector<double> adj_signature(const lpm_ctx *c, const double *rec, int R, double bandwidth,
                                  int every)
{
    std::vector<double> sig(rec, rec + 3 * (size_t)R);
    sig.push_back(bandwidth);
    sig.push_back(every);
    sig.push_back((double)c->params_version);
    sig.push_back(c->adj_traj ? 1.0 : 0.0);
    sig.push_back(c->adj_sorted ? 1.0 : 0.0);
    return sig;
}

lpm_status adj_forward(lpm_ctx *c, const double *rec, int R, double bandwidth, int every,
                       AdjParams &A, StepParams &P)
{
    lpm_status st = adj_prepare(c, rec, R, bandwidth, every, A, P);
    if (st != LPM_OK) return st;
    LPM_CUDA(c, cudaMemsetAsync(c->d_rC, 0, (size_t)c->cfg.n_scenarios * R * sizeof(double), c->stream));
    if (c->adj_sorted) {
        st = adj_forward_sorted(c, P, A);
        if (st != LPM_OK) return st;
    } else {
        LPM_CUDA(c, launch_adj_forward(c->stream, P, A, (int)c->adj_tiles.size()));
        c->n_launches++;
    }
    st = check_device_error(c);
    if (st != LPM_OK) return st;
    c->adj_sig = adj_signature(c, rec, R, bandwidth, every);
    return LPM_OK;
}

}  // namespace

lpm_status lpm_receptors(lpm_ctx *c, const double *rec, int R, double bandwidth, int sample_every,
                         double *C)
{
    if (!c) return LPM_E_INVALID;
    NvtxRange nr("lpm_receptors (adjoint forward)");
    if (!C) return fail(c, LPM_E_INVALID, "C is NULL");
    AdjParams A;
    StepParams P;
    lpm_status st = adj_forward(c, rec, R, bandwidth, sample_every, A, P);
    if (st != LPM_OK) return st;
    LPM_CUDA(c, cudaMemcpy(C, c->d_rC, (size_t)c->cfg.n_scenarios * R * sizeof(double),
                           cudaMemcpyDeviceToHost));
    return LPM_OK;
}

lpm_status lpm_adjoint(lpm_ctx *c, const double *rec, int R, double bandwidth, int sample_every,
                       const double *dL_dC, double *grad)
{
    if (!c) return LPM_E_INVALID;
    NvtxRange nr("lpm_adjoint (reverse sweep)");
    if (!dL_dC || !grad) return fail(c, LPM_E_INVALID, "dL_dC and grad are required");
    AdjParams A;
    StepParams P;
    lpm_status st;
    if (c->adj_sig != adj_signature(c, rec, R, bandwidth, sample_every)) {
        st = adj_forward(c, rec, R, bandwidth, sample_every, A, P);   // states for the sweep
    } else {
        st = adj_prepare(c, rec, R, bandwidth, sample_every, A, P, true);
    }
    if (st != LPM_OK) return st;
    const size_t ns = (size_t)c->cfg.n_scenarios;
    for (size_t i = 0; i < ns * (size_t)R; ++i)
        if (!is_finite(dL_dC[i])) return fail(c, LPM_E_INVALID, "dL_dC not finite");
    LPM_CUDA(c, cudaMemcpyAsync(c->d_rw, dL_dC, ns * R * sizeof(double), cudaMemcpyHostToDevice,
                                c->stream));
    LPM_CUDA(c, cudaMemsetAsync(c->d_rgrad, 0, ns * A.ng * sizeof(double), c->stream));
    if (c->adj_sorted) {
        st = adj_backward_sorted(c, P, A);
        if (st != LPM_OK) return st;
    } else {
        LPM_CUDA(c, launch_adj_backward(c->stream, P, A, (int)c->adj_tiles.size()));
        c->n_launches++;
    }
    st = check_device_error(c);
    if (st != LPM_OK) return st;
    LPM_CUDA(c, cudaMemcpy(grad, c->d_rgrad, ns * A.ng * sizeof(double), cudaMemcpyDeviceToHost));
    return LPM_OK;
}

lpm_status lpm_set_adjoint_storage(lpm_ctx *c, uint64_t max_bytes)
{
    if (!c) return LPM_E_INVALID;
    c->adj_store_max = (size_t)max_bytes;
    c->adj_sig.clear();
    return LPM_OK;
}

lpm_status lpm_adjoint_storage(lpm_ctx *c, int *trajectory, uint64_t *bytes)
{
    if (!c || !trajectory || !bytes) return LPM_E_INVALID;
    *trajectory = c->adj_traj ? 1 : 0;
    *bytes = (uint64_t)((c->d_traj_cap + c->d_fin_cap + c->d_ckpt_cap) * sizeof(float4));
    return LPM_OK;
}

// ---- checkpoint / resume --------------------------------------------------------
namespace {
struct SaveHeader {
    char magic[8];               // "LPMSAVE4"
    long long k, n_bins, n_slots, n_scen, ncell, ndep, n_ctr;
    long long dose_every, n_dose; // dosage interval (0: none saved) and samples taken
    long long n_species;          // decay-chain species (daughters' grids saved when > 1)
    long long langevin;           // the Langevin w' of every slot follows when 1
};
}  // namespace

lpm_status lpm_save(lpm_ctx *c, void *buf, size_t *n)
{
    if (!c || !n) return LPM_E_INVALID;
    const size_t ns = (size_t)c->cfg.n_scenarios;
    const bool dose = c->d_dose && c->dose_every > 0;
    const size_t bytes = sizeof(SaveHeader) + (size_t)c->n_slots_used * sizeof(float4) +
                         ns * (c->ncell() + c->ndep()) * sizeof(unsigned long long) +
                         (size_t)N_COUNTERS * ns * sizeof(unsigned long long) +
                         (dose ? ns * c->ncell() * sizeof(unsigned long long) : 0) +
                         (size_t)(c->n_species - 1) * ns * (c->ncell() + c->ndep()) * 8 +
                         (c->langevin ? (size_t)c->n_slots_used * sizeof(float) : 0);
    if (!buf) {
        *n = bytes;
        return LPM_OK;
    }
    if (*n < bytes) return fail(c, LPM_E_INVALID, "buffer holds %zu bytes, %zu needed", *n, bytes);
    lpm_status st = check_device_error(c);
    if (st != LPM_OK) return st;
    SaveHeader h;
    std::memcpy(h.magic, "LPMSAVE4", 8);
    h.k = c->k;
    h.n_bins = c->n_bins;
    h.n_slots = c->n_slots_used;
    h.n_scen = (long long)ns;
    h.ncell = (long long)c->ncell();
    h.ndep = (long long)c->ndep();
    h.n_ctr = N_COUNTERS;
    h.dose_every = dose ? c->dose_every : 0;
    h.n_dose = dose ? c->n_dose : 0;
    h.n_species = c->n_species;
    h.langevin = c->langevin;
    char *o = static_cast<char *>(buf);
    std::memcpy(o, &h, sizeof h);
    o += sizeof h;
    // particles in slot order (the sorted layout is not part of the state)
    const size_t sb = (size_t)c->n_slots_used * sizeof(float4);
    if (c->d_sorted[0]) {
        float4 *tmp = c->d_sorted[1 - c->cur];
        {
            const lpm_status sm = ensure_slot_map(c);
            if (sm != LPM_OK) return sm;
        }
        LPM_CUDA(c, launch_gather(c->stream, c->d_state, c->d_sorted[c->cur], c->d_slot_of,
                                  c->d_grave, 0, c->n_slots_used, tmp));
        LPM_CUDA(c, cudaMemcpyAsync(o, tmp, sb, cudaMemcpyDeviceToHost, c->stream));
        c->n_launches++;
    } else {
        LPM_CUDA(c, cudaMemcpyAsync(o, c->d_state, sb, cudaMemcpyDeviceToHost, c->stream));
    }
    o += sb;
    LPM_CUDA(c, cudaMemcpyAsync(o, c->d_conc, ns * c->ncell() * 8, cudaMemcpyDeviceToHost, c->stream));
    o += ns * c->ncell() * 8;
    LPM_CUDA(c, cudaMemcpyAsync(o, c->d_dep, ns * c->ndep() * 8, cudaMemcpyDeviceToHost, c->stream));
    o += ns * c->ndep() * 8;
    LPM_CUDA(c, cudaMemcpyAsync(o, c->d_ctr, ns * N_COUNTERS * 8, cudaMemcpyDeviceToHost, c->stream));
    o += ns * N_COUNTERS * 8;
    if (dose) {
        LPM_CUDA(c, cudaMemcpyAsync(o, c->d_dose, ns * c->ncell() * 8, cudaMemcpyDeviceToHost,
                                    c->stream));
        o += ns * c->ncell() * 8;
    }
    if (c->n_species > 1) {
        const size_t nd = (size_t)(c->n_species - 1) * ns;
        LPM_CUDA(c, cudaMemcpyAsync(o, c->d_sp_conc, nd * c->ncell() * 8, cudaMemcpyDeviceToHost,
                                    c->stream));
        o += nd * c->ncell() * 8;
        LPM_CUDA(c, cudaMemcpyAsync(o, c->d_sp_dep, nd * c->ndep() * 8, cudaMemcpyDeviceToHost,
                                    c->stream));
        o += nd * c->ndep() * 8;
    }
    if (c->langevin) {
        // the spare sorted-w buffer is free here (the gather of the particles above used
        // the spare state buffer)
        float *tmp = c->d_w_sorted[1 - c->cur];
        {
            const lpm_status sm = ensure_slot_map(c);
            if (sm != LPM_OK) return sm;
        }
        LPM_CUDA(c, launch_gather_w(c->stream, c->d_w_home, c->d_w_sorted[c->cur], c->d_slot_of, 0,
                                    c->n_slots_used, tmp));
        LPM_CUDA(c, cudaMemcpyAsync(o, tmp, (size_t)c->n_slots_used * sizeof(float),
                                    cudaMemcpyDeviceToHost, c->stream));
    }
    LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    *n = bytes;
    return LPM_OK;
}

lpm_status lpm_load(lpm_ctx *c, const void *buf, size_t n)
{
    if (!c || !buf) return LPM_E_INVALID;
    if (c->n_released != c->cfg.n_scenarios)
        return fail(c, LPM_E_STATE, "release every scenario before loading a saved run");
    SaveHeader h;
    if (n < sizeof h) return fail(c, LPM_E_INVALID, "buffer too small for a saved run");
    std::memcpy(&h, buf, sizeof h);
    const size_t ns = (size_t)c->cfg.n_scenarios;
    if (std::memcmp(h.magic, "LPMSAVE4", 8) != 0 || h.n_slots != c->n_slots_used ||
        h.n_species != c->n_species || h.langevin != c->langevin ||
        h.n_scen != (long long)ns || h.ncell != (long long)c->ncell() ||
        h.ndep != (long long)c->ndep() || h.n_ctr != N_COUNTERS || h.k < 0 ||
        h.k > c->cfg.n_steps || h.dose_every < 0 || h.dose_every > 0x7fffffffLL)
        return fail(c, LPM_E_INVALID, "saved run does not match this context");
    // a snapshot is taken at most once per step, a dosage sample once per dose_every steps
    if (h.n_bins < 0 || h.n_bins > h.k || h.n_dose < 0 ||
        (h.dose_every > 0 ? h.n_dose > h.k / h.dose_every : h.n_dose != 0))
        return fail(c, LPM_E_INVALID, "saved run has inconsistent snapshot or dosage counts");
    const size_t sb = (size_t)c->n_slots_used * sizeof(float4);
    const size_t need = sizeof h + sb + ns * (c->ncell() + c->ndep() + N_COUNTERS) * 8 +
                        (h.dose_every > 0 ? ns * c->ncell() * 8 : 0) +
                        (size_t)(c->n_species - 1) * ns * (c->ncell() + c->ndep()) * 8 +
                        (c->langevin ? (size_t)c->n_slots_used * sizeof(float) : 0);
    if (n < need) return fail(c, LPM_E_INVALID, "saved run truncated (%zu of %zu bytes)", n, need);
    lpm_status st;
    if (h.dose_every > 0) {
        // the dosage grid may need an allocation: take it before any particle, grid or
        // counter is overwritten, so that a failed allocation leaves the run as it was
        st = lpm_set_dosage(c, (int)h.dose_every);
        if (st != LPM_OK) return st;
    }
    st = upload_tables(c);
    if (st != LPM_OK) return st;
    const char *i = static_cast<const char *>(buf) + sizeof h;
    LPM_CUDA(c, cudaMemcpyAsync(c->d_state, i, sb, cudaMemcpyHostToDevice, c->stream));
    i += sb;
    LPM_CUDA(c, cudaMemcpyAsync(c->d_conc, i, ns * c->ncell() * 8, cudaMemcpyHostToDevice, c->stream));
    i += ns * c->ncell() * 8;
    LPM_CUDA(c, cudaMemcpyAsync(c->d_dep, i, ns * c->ndep() * 8, cudaMemcpyHostToDevice, c->stream));
    i += ns * c->ndep() * 8;
    LPM_CUDA(c, cudaMemcpyAsync(c->d_ctr, i, ns * N_COUNTERS * 8, cudaMemcpyHostToDevice, c->stream));
    i += ns * N_COUNTERS * 8;
    if (h.dose_every > 0) {
        // the grid was allocated above; the counters copied above hold the saved dose_out row
        LPM_CUDA(c, cudaMemcpyAsync(c->d_dose, i, ns * c->ncell() * 8, cudaMemcpyHostToDevice,
                                    c->stream));
        c->n_dose = h.n_dose;
        i += ns * c->ncell() * 8;
    } else if (c->d_dose) {
        st = lpm_set_dosage(c, 0);
        if (st != LPM_OK) return st;
    }
    if (c->n_species > 1) {
        const size_t nd = (size_t)(c->n_species - 1) * ns;
        LPM_CUDA(c, cudaMemcpyAsync(c->d_sp_conc, i, nd * c->ncell() * 8, cudaMemcpyHostToDevice,
                                    c->stream));
        i += nd * c->ncell() * 8;
        LPM_CUDA(c, cudaMemcpyAsync(c->d_sp_dep, i, nd * c->ndep() * 8, cudaMemcpyHostToDevice,
                                    c->stream));
        i += nd * c->ndep() * 8;
    }
    if (c->langevin)
        LPM_CUDA(c, cudaMemcpyAsync(c->d_w_home, i, (size_t)c->n_slots_used * sizeof(float),
                                    cudaMemcpyHostToDevice, c->stream));
    LPM_CUDA(c, cudaMemsetAsync(c->d_err, 0, sizeof(unsigned int), c->stream));
    st = clear_sort_state(c, false);     // every particle at its home slot
    if (st != LPM_OK) return st;
    LPM_CUDA(c, cudaStreamSynchronize(c->stream));
    c->k = h.k;
    c->n_bins = h.n_bins;
    return LPM_OK;
}

lpm_status lpm_draws(uint64_t seed, const uint64_t *pid, const uint32_t *step, uint32_t stream,
                     int64_t n, uint32_t *words, float *normals)
{
    g_create_error.clear();
    if (n < 0 || (n > 0 && (!pid || !step || !words || !normals)))
        return fail(nullptr, LPM_E_INVALID, "lpm_draws: invalid arguments");
    if (n == 0) return LPM_OK;
    unsigned long long *d_pid = nullptr;
    unsigned int *d_step = nullptr;
    uint4 *d_w = nullptr;
    float *d_n = nullptr;
    lpm_status st = LPM_OK;
    cudaError_t e = cudaMalloc(&d_pid, n * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMalloc(&d_step, n * sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMalloc(&d_w, n * sizeof(uint4));
    if (e == cudaSuccess) e = cudaMalloc(&d_n, n * 3 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(d_pid, pid, n * sizeof(unsigned long long), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_step, step, n * sizeof(unsigned int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = launch_draws(nullptr, seed, d_pid, d_step, stream, n, d_w, d_n);
    if (e == cudaSuccess) e = cudaMemcpy(words, d_w, n * sizeof(uint4), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(normals, d_n, n * 3 * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        st = fail(nullptr, e == cudaErrorMemoryAllocation ? LPM_E_OOM : LPM_E_CUDA, "lpm_draws: %s",
                  cudaGetErrorString(e));
    }
    cudaFree(d_pid);
    cudaFree(d_step);
    cudaFree(d_w);
    cudaFree(d_n);
    return st;
}

}  // extern "C"
