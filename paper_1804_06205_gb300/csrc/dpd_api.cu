// C ABI of libdpd (include/dpd.h): argument validation, the bond table in
// CSR form, and dispatch to the FP32 or FP64 batch engine.  A dpd_handle is a
// batch holding exactly one system.
#include <cmath>
#include <cstring>
#include <memory>
#include <new>
#include <string>

#include "dpd.h"
#include "engine.h"

struct dpd_handle {
    std::unique_ptr<dpd::BatchBase> eng;
    std::string err;
    int64_t n = 0;
    int32_t nc[3] = {0, 0, 0};
    int slot = 0;
};

struct dpd_batch {
    std::unique_ptr<dpd::BatchBase> eng;
    std::string err;
    dpd_options opt;
};

namespace {

bool is_fin(double x) { return std::isfinite(x); }

int fail(std::string &err, int code, const char *msg) {
    err = msg;
    return code;
}

thread_local std::string g_create_err;

int add_bonds(const dpd::Config &c, const dpd_bond *b, int64_t nb, std::vector<int64_t> &deg) {
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

// Validate one system's parameters into a Config; returns DPD_OK or
// DPD_EINVAL with *why set.
int build_config(const dpd_box *box, int64_t n, const int32_t *types, int32_t ntypes,
                 const double *a_ij, double gamma, double kT, double dt, const dpd_bond *bonds,
                 int64_t nbonds, const dpd_bond *morse, int64_t nmorse, double lambda,
                 uint64_t seed, int32_t noise, int32_t tile_cells, dpd::Config &c,
                 const char **why) {
    auto bad = [why](const char *m) {
        *why = m;
        return DPD_EINVAL;
    };
    if (!box) return bad("box is NULL");
    if (n <= 0 || n > (int64_t)1 << 30) return bad("n out of range");
    if (!types || !a_ij) return bad("types or a_ij is NULL");
    if (ntypes < 1 || ntypes > 16) return bad("ntypes must be in [1, 16]");
    if (!is_fin(gamma) || !is_fin(kT) || !is_fin(dt) || gamma < 0 || kT < 0 || dt <= 0)
        return bad("gamma, kT must be >= 0 and dt > 0");
    if (!is_fin(lambda)) return bad("lambda not finite");
    if (noise != DPD_NOISE_GAUSS && noise != DPD_NOISE_UNIFORM) return bad("bad noise");
    // cells per edge and their product are checked before any conversion or
    // multiplication could overflow: each factor is at most 2^31 - 2 and the
    // running product never exceeds it either
    const int64_t kMaxCells = ((int64_t)1 << 31) - 2;
    int64_t ncell = 1;
    for (int k = 0; k < 3; ++k) {
        const double L = box->L[k];
        if (!is_fin(L) || L < 3.0) return bad("every box edge must be >= 3");
        const double nc = std::floor(L);
        if (nc > (double)kMaxCells) return bad("too many cells");
        ncell *= (int64_t)nc;
        if (ncell > kMaxCells) return bad("too many cells");
        c.L[k] = L;
        c.nc[k] = (int32_t)nc;
        c.h[k] = L / nc;
        c.inv_h[k] = nc / L;
    }
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
    c.lambda = lambda;
    c.seed = seed;
    c.noise = noise;
    c.tile_cells = tile_cells;
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
    return DPD_OK;
}

dpd::BatchBase *make_engine(const dpd::BatchConfig &bc, int precision, int *rc,
                            std::string *err) {
    return precision == DPD_FP64 ? dpd::make_batch_f64(bc, rc, err)
                                 : dpd::make_batch_f32(bc, rc, err);
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
    opt->use_graph = 0;
    opt->persistent = 0;
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
    if (o.precision != DPD_FP32 && o.precision != DPD_FP64) {
        g_create_err = "bad precision";
        return DPD_EINVAL;
    }
    dpd::Config c;
    const char *why = "";
    int rc = build_config(box, n, types, ntypes, a_ij, gamma, kT, dt, bonds, nbonds, morse,
                          nmorse, o.lambda, o.seed, o.noise, o.tile_cells, c, &why);
    if (rc) {
        g_create_err = why;
        return rc;
    }
    dpd::BatchConfig bc;
    bc.max_beads = n;
    bc.max_cells = (int64_t)c.nc[0] * c.nc[1] * c.nc[2];
    bc.max_bonds = (int64_t)c.bpartner.size();
    bc.max_systems = 1;
    bc.threads = o.threads;
    bc.sample_every = o.sample_every < 0 ? 0 : o.sample_every;
    bc.use_graph = o.use_graph != 0;
    bc.persistent = o.persistent != 0;
    bc.stream = o.cuda_stream;
    dpd_handle *h = new (std::nothrow) dpd_handle();
    if (!h) return DPD_ENOMEM;
    h->n = n;
    for (int k = 0; k < 3; ++k) h->nc[k] = c.nc[k];
    std::string err;
    dpd::BatchBase *e = make_engine(bc, o.precision, &rc, &err);
    if (!e) {
        g_create_err = err;
        delete h;
        return rc ? rc : DPD_ECUDA;
    }
    h->eng.reset(e);
    rc = e->add_system(c, &h->slot);
    if (rc) {
        g_create_err = e->last_error();
        delete h;
        return rc;
    }
    *out = h;
    return DPD_OK;
}

int dpd_set_state(dpd_handle *h, const double *pos, const double *vel, int64_t step) {
    if (!h) return DPD_EINVAL;
    if (!pos || !vel) return fail(h->err, DPD_EINVAL, "pos or vel is NULL");
    h->err.clear();
    return h->eng->set_state(h->slot, pos, vel, step);
}

int dpd_step(dpd_handle *h, int64_t nsteps) {
    if (!h) return DPD_EINVAL;
    return h->eng->step(nsteps);
}

int dpd_get_state(dpd_handle *h, double *pos, double *vel, double *force, int64_t *step) {
    if (!h) return DPD_EINVAL;
    return h->eng->get_state(h->slot, pos, vel, force, step);
}

int dpd_observables(dpd_handle *h, dpd_obs *out) {
    if (!h || !out) return DPD_EINVAL;
    return h->eng->observables(h->slot, out);
}

int dpd_gr(dpd_handle *h, double rmax, int32_t nbins, uint64_t *counts) {
    if (!h) return DPD_EINVAL;
    return h->eng->gr(h->slot, rmax, nbins, counts);
}

int dpd_get_cells(dpd_handle *h, uint32_t *key_by_id, int64_t *order, int64_t *cell_start) {
    if (!h) return DPD_EINVAL;
    return h->eng->get_cells(h->slot, key_by_id, order, cell_start);
}

int dpd_checkpoint_bytes(const dpd_handle *h, int64_t *bytes) {
    if (!h || !bytes) return DPD_EINVAL;
    *bytes = h->eng->checkpoint_bytes(h->slot);
    return DPD_OK;
}

int dpd_get_checkpoint(dpd_handle *h, void *buf, int64_t bytes) {
    if (!h) return DPD_EINVAL;
    return h->eng->get_checkpoint(h->slot, buf, bytes);
}

int dpd_set_checkpoint(dpd_handle *h, const void *buf, int64_t bytes) {
    if (!h) return DPD_EINVAL;
    h->err.clear();
    return h->eng->set_checkpoint(h->slot, buf, bytes);
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

// ---------------------------------------------------------------- batches
int dpd_batch_create(const dpd_batch_capacity *cap, const dpd_options *opt, dpd_batch **out) {
    g_create_err.clear();
    if (!out || !cap) return DPD_EINVAL;
    *out = nullptr;
    if (cap->max_beads <= 0 || cap->max_beads > (int64_t)1 << 30 || cap->max_cells <= 0 ||
        cap->max_cells > ((int64_t)1 << 31) - 2 || cap->max_bonds < 0 ||
        cap->max_bonds > (int64_t)1 << 29 || cap->max_systems <= 0 ||
        cap->max_systems > 65536) {
        g_create_err = "capacity out of range";
        return DPD_EINVAL;
    }
    dpd_batch *b = new (std::nothrow) dpd_batch();
    if (!b) return DPD_ENOMEM;
    dpd_default_options(&b->opt);
    if (opt) b->opt = *opt;
    if (b->opt.precision != DPD_FP32 && b->opt.precision != DPD_FP64) {
        delete b;
        g_create_err = "bad precision";
        return DPD_EINVAL;
    }
    dpd::BatchConfig bc;
    bc.max_beads = cap->max_beads;
    bc.max_cells = cap->max_cells;
    bc.max_bonds = 2 * cap->max_bonds;
    bc.max_systems = cap->max_systems;
    bc.threads = b->opt.threads;
    bc.sample_every = 0;
    bc.use_graph = b->opt.use_graph != 0;
    bc.persistent = b->opt.persistent != 0;
    bc.stream = b->opt.cuda_stream;
    int rc = DPD_OK;
    std::string err;
    dpd::BatchBase *e = make_engine(bc, b->opt.precision, &rc, &err);
    if (!e) {
        g_create_err = err;
        delete b;
        return rc ? rc : DPD_ECUDA;
    }
    b->eng.reset(e);
    *out = b;
    return DPD_OK;
}

int dpd_batch_add(dpd_batch *b, const dpd_box *box, int64_t n, const int32_t *types,
                  int32_t ntypes, const double *a_ij, double gamma, double kT, double dt,
                  const dpd_bond *bonds, int64_t nbonds, const dpd_bond *morse, int64_t nmorse,
                  double lambda, uint64_t seed, int32_t tile_cells, const double *pos,
                  const double *vel, int64_t step, int32_t *sys) {
    if (!b || !sys) return DPD_EINVAL;
    if (!pos || !vel) return fail(b->err, DPD_EINVAL, "pos or vel is NULL");
    dpd::Config c;
    const char *why = "";
    int rc = build_config(box, n, types, ntypes, a_ij, gamma, kT, dt, bonds, nbonds, morse,
                          nmorse, lambda, seed, b->opt.noise,
                          tile_cells > 0 ? tile_cells : b->opt.tile_cells, c, &why);
    if (rc) return fail(b->err, rc, why);
    int slot = -1;
    rc = b->eng->add_system(c, &slot);
    if (rc) return fail(b->err, rc, b->eng->last_error());
    rc = b->eng->set_state(slot, pos, vel, step);
    if (rc) {
        b->err = b->eng->last_error();
        b->eng->remove_system(slot);
        return rc;
    }
    *sys = slot;
    b->err.clear();
    return DPD_OK;
}

int dpd_batch_remove(dpd_batch *b, int32_t sys) {
    if (!b) return DPD_EINVAL;
    return b->eng->remove_system(sys);
}

int dpd_batch_step(dpd_batch *b, int64_t nsteps) {
    if (!b) return DPD_EINVAL;
    return b->eng->step(nsteps);
}

int dpd_batch_get_state(dpd_batch *b, int32_t sys, double *pos, double *vel, double *force,
                        int64_t *step) {
    if (!b) return DPD_EINVAL;
    return b->eng->get_state(sys, pos, vel, force, step);
}

int dpd_batch_observables(dpd_batch *b, int32_t sys, dpd_obs *out) {
    if (!b || !out) return DPD_EINVAL;
    return b->eng->observables(sys, out);
}

int dpd_batch_usage(const dpd_batch *b, int64_t used[4], int64_t cap[4], int32_t *nsys) {
    if (!b) return DPD_EINVAL;
    int64_t u[4], c[4];
    b->eng->usage(u, c);
    for (int k = 0; k < 4; ++k) {
        if (used) used[k] = u[k];
        if (cap) cap[k] = c[k];
    }
    if (nsys) *nsys = b->eng->nlive();
    return DPD_OK;
}

int dpd_batch_checkpoint_bytes(const dpd_batch *b, int32_t sys, int64_t *bytes) {
    if (!b || !bytes) return DPD_EINVAL;
    *bytes = b->eng->checkpoint_bytes(sys);
    return *bytes > 0 ? DPD_OK : DPD_EINVAL;
}

int dpd_batch_get_checkpoint(dpd_batch *b, int32_t sys, void *buf, int64_t bytes) {
    if (!b) return DPD_EINVAL;
    return b->eng->get_checkpoint(sys, buf, bytes);
}

int dpd_batch_set_checkpoint(dpd_batch *b, int32_t sys, const void *buf, int64_t bytes) {
    if (!b) return DPD_EINVAL;
    b->err.clear();
    return b->eng->set_checkpoint(sys, buf, bytes);
}

int dpd_batch_sync(dpd_batch *b) {
    if (!b) return DPD_EINVAL;
    return b->eng->sync();
}

int64_t dpd_batch_launch_count(const dpd_batch *b) { return b ? b->eng->launches() : 0; }

int dpd_batch_profile_begin(dpd_batch *b, int64_t max_steps) {
    if (!b || max_steps < 1 || max_steps > 100000) return DPD_EINVAL;
    return b->eng->profile_begin(max_steps);
}

int dpd_batch_profile_end(dpd_batch *b, double ms[3], int64_t *nsteps) {
    if (!b || !ms) return DPD_EINVAL;
    return b->eng->profile_end(ms, nsteps);
}

const char *dpd_batch_last_error(const dpd_batch *b) {
    if (!b) return g_create_err.c_str();
    if (!b->err.empty()) return b->err.c_str();
    return b->eng ? b->eng->last_error() : "";
}

int dpd_batch_destroy(dpd_batch *b) {
    delete b;
    return DPD_OK;
}

}  // extern "C"
