// C ABI of libdpd (include/dpd.h): argument validation, the bond table in
// CSR form, and dispatch to the FP32 or FP64 engine.
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "dpd.h"
#include "engine.h"

struct dpd_handle {
    std::unique_ptr<dpd::EngineBase> eng;
    std::string err;
    int64_t n = 0;
    int32_t nc[3] = {0, 0, 0};
};

namespace {

bool is_fin(double x) { return std::isfinite(x); }

int fail(dpd_handle *h, int code, const char *msg) {
    if (h) h->err = msg;
    return code;
}

thread_local std::string g_create_err;

int add_bonds(dpd::Config &c, const dpd_bond *b, int64_t nb, std::vector<int64_t> &deg) {
    if (nb < 0 || (nb > 0 && !b)) return DPD_EINVAL;
    for (int64_t k = 0; k < nb; ++k) {
        const dpd_bond &r = b[k];
        if (r.i < 0 || r.j < 0 || r.i >= c.n || r.j >= c.n || r.i == r.j) return DPD_EINVAL;
        if (r.kind < DPD_BOND_HARMONIC || r.kind > DPD_BOND_MORSE) return DPD_EINVAL;
        if (!is_fin(r.r0) || !is_fin(r.k) || !is_fin(r.alpha) || r.r0 < 0) return DPD_EINVAL;
        deg[r.i]++;
        deg[r.j]++;
    }
    return DPD_OK;
}

void fill_bonds(dpd::Config &c, const dpd_bond *b, int64_t nb, std::vector<int32_t> &fillp) {
    for (int64_t k = 0; k < nb; ++k) {
        const dpd_bond &r = b[k];
        const int32_t ends[2][2] = {{r.i, r.j}, {r.j, r.i}};
        for (auto &e : ends) {
            const int32_t slot = fillp[e[0]]++;
            c.bpartner[slot] = e[1];
            c.bkind[slot] = r.kind;
            c.br0[slot] = r.r0;
            c.bk[slot] = r.k;
            c.balpha[slot] = r.alpha;
        }
    }
}

}  // namespace

extern "C" {

void dpd_default_options(dpd_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->lambda = 0.65;
    opt->seed = 0;
    opt->precision = DPD_FP32;
    opt->noise = DPD_NOISE_GAUSS;
    opt->sample_every = 0;
    opt->tile_cells = 0;
    opt->threads = 0;
    opt->use_graph = 1;
    opt->cuda_stream = nullptr;
}

int dpd_create(const dpd_box *box, int64_t n, const int32_t *types, int32_t ntypes,
               const double *a_ij, double gamma, double kT, double dt, const dpd_bond *bonds,
               int64_t nbonds, const dpd_bond *morse, int64_t nmorse, const dpd_options *opt,
               dpd_handle **out) {
    g_create_err.clear();
    if (!out) return DPD_EINVAL;
    *out = nullptr;
    dpd_options o;
    dpd_default_options(&o);
    if (opt) o = *opt;
    auto bad = [](const char *m) {
        g_create_err = m;
        return DPD_EINVAL;
    };
    if (!box) return bad("box is NULL");
    if (n <= 0 || n > (int64_t)1 << 30) return bad("n out of range");
    if (!types || !a_ij) return bad("types or a_ij is NULL");
    if (ntypes < 1 || ntypes > 16) return bad("ntypes must be in [1, 16]");
    if (!is_fin(gamma) || !is_fin(kT) || !is_fin(dt) || gamma < 0 || kT < 0 || dt <= 0)
        return bad("gamma, kT must be >= 0 and dt > 0");
    if (!is_fin(o.lambda)) return bad("lambda not finite");
    if (o.precision != DPD_FP32 && o.precision != DPD_FP64) return bad("bad precision");
    if (o.noise != DPD_NOISE_GAUSS && o.noise != DPD_NOISE_UNIFORM) return bad("bad noise");
    dpd::Config c;
    int64_t ncell = 1;
    for (int k = 0; k < 3; ++k) {
        const double L = box->L[k];
        if (!is_fin(L) || L < 3.0) return bad("every box edge must be >= 3");
        const double nc = std::floor(L);
        c.L[k] = L;
        c.nc[k] = (int32_t)nc;
        c.h[k] = L / nc;
        c.inv_h[k] = nc / L;
        ncell *= (int64_t)nc;
    }
    if (ncell > ((int64_t)1 << 31) - 2) return bad("too many cells");
    c.n = n;
    c.ntypes = ntypes;
    c.types.assign(types, types + n);
    for (int64_t i = 0; i < n; ++i)
        if (types[i] < 0 || types[i] >= ntypes) return bad("type out of range");
    c.a.assign(a_ij, a_ij + (size_t)ntypes * ntypes);
    for (int p = 0; p < ntypes; ++p)
        for (int q = 0; q < ntypes; ++q)
            if (!is_fin(a_ij[p * ntypes + q]) || a_ij[p * ntypes + q] != a_ij[q * ntypes + p])
                return bad("a_ij must be finite and symmetric");
    c.gamma = gamma;
    c.kT = kT;
    c.dt = dt;
    c.lambda = o.lambda;
    c.seed = o.seed;
    c.noise = o.noise;
    c.sample_every = o.sample_every < 0 ? 0 : o.sample_every;
    c.tile_cells = o.tile_cells;
    c.threads = o.threads;
    c.use_graph = o.use_graph != 0;
    c.stream = o.cuda_stream;
    std::vector<int64_t> deg((size_t)n, 0);
    if (add_bonds(c, bonds, nbonds, deg) || add_bonds(c, morse, nmorse, deg))
        return bad("bad bond record");
    c.nbonds = nbonds + nmorse;
    c.bptr.assign((size_t)n + 1, 0);
    for (int64_t i = 0; i < n; ++i) c.bptr[i + 1] = c.bptr[i] + (int32_t)deg[i];
    const size_t nrec = (size_t)c.bptr[n];
    c.bpartner.resize(nrec);
    c.bkind.resize(nrec);
    c.br0.resize(nrec);
    c.bk.resize(nrec);
    c.balpha.resize(nrec);
    std::vector<int32_t> fillp(c.bptr.begin(), c.bptr.end() - 1);
    fill_bonds(c, bonds, nbonds, fillp);
    fill_bonds(c, morse, nmorse, fillp);

    dpd_handle *h = new (std::nothrow) dpd_handle();
    if (!h) return DPD_ENOMEM;
    h->n = n;
    for (int k = 0; k < 3; ++k) h->nc[k] = c.nc[k];
    int rc = DPD_OK;
    std::string err;
    dpd::EngineBase *e = o.precision == DPD_FP64 ? dpd::make_engine_f64(c, &rc, &err)
                                                 : dpd::make_engine_f32(c, &rc, &err);
    if (!e) {
        g_create_err = err;
        delete h;
        return rc ? rc : DPD_ECUDA;
    }
    h->eng.reset(e);
    *out = h;
    return DPD_OK;
}

int dpd_set_state(dpd_handle *h, const double *pos, const double *vel, int64_t step) {
    if (!h) return DPD_EINVAL;
    if (!pos || !vel) return fail(h, DPD_EINVAL, "pos or vel is NULL");
    h->err.clear();
    return h->eng->set_state(pos, vel, step);
}

int dpd_step(dpd_handle *h, int64_t nsteps) {
    if (!h) return DPD_EINVAL;
    return h->eng->step(nsteps);
}

int dpd_get_state(dpd_handle *h, double *pos, double *vel, double *force, int64_t *step) {
    if (!h) return DPD_EINVAL;
    return h->eng->get_state(pos, vel, force, step);
}

int dpd_observables(dpd_handle *h, dpd_obs *out) {
    if (!h || !out) return DPD_EINVAL;
    return h->eng->observables(out);
}

int dpd_gr(dpd_handle *h, double rmax, int32_t nbins, uint64_t *counts) {
    if (!h) return DPD_EINVAL;
    return h->eng->gr(rmax, nbins, counts);
}

int dpd_get_cells(dpd_handle *h, uint32_t *key_by_id, int64_t *order, int64_t *cell_start) {
    if (!h) return DPD_EINVAL;
    return h->eng->get_cells(key_by_id, order, cell_start);
}

int dpd_cell_dims(const dpd_handle *h, int64_t nc[3]) {
    if (!h || !nc) return DPD_EINVAL;
    for (int k = 0; k < 3; ++k) nc[k] = h->nc[k];
    return DPD_OK;
}

int dpd_sync(dpd_handle *h) {
    if (!h) return DPD_EINVAL;
    return h->eng->sync();
}

int64_t dpd_launch_count(const dpd_handle *h) { return h ? h->eng->launches() : 0; }

int dpd_profile_begin(dpd_handle *h, int64_t max_steps) {
    if (!h || max_steps < 1 || max_steps > 100000) return DPD_EINVAL;
    return h->eng->profile_begin(max_steps);
}

int dpd_profile_end(dpd_handle *h, double ms[3], int64_t *nsteps) {
    if (!h || !ms) return DPD_EINVAL;
    return h->eng->profile_end(ms, nsteps);
}

int dpd_destroy(dpd_handle *h) {
    delete h;
    return DPD_OK;
}

const char *dpd_strerror(int code) {
    switch (code) {
        case DPD_OK: return "ok";
        case DPD_EINVAL: return "invalid argument";
        case DPD_ENOMEM: return "out of memory";
        case DPD_ECUDA: return "CUDA runtime error";
        case DPD_EUNSTABLE: return "non-finite state (unstable integration)";
        case DPD_ETIMEOUT: return "a bounded device wait gave up";
        case DPD_ENOSTATE: return "no state set (call dpd_set_state first)";
        default: return "unknown error";
    }
}

const char *dpd_last_error(const dpd_handle *h) {
    if (!h) return g_create_err.c_str();
    if (!h->err.empty()) return h->err.c_str();
    return h->eng ? h->eng->last_error() : "";
}

}  // extern "C"
