// Host-side interface between the C ABI (dpd_api.cu) and the per-precision
// engines (engine_f32.cu, engine_f64.cu).  No device code here.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "dpd.h"

namespace dpd {

// Everything dpd_create validated, in the layout the engines upload.
struct Config {
    double L[3];
    int64_t n;
    int32_t ntypes;
    std::vector<int32_t> types;      // [n]
    std::vector<double> a;           // [ntypes*ntypes]
    double gamma, kT, dt, lambda;
    uint64_t seed;
    int32_t noise;
    int32_t sample_every;
    int32_t tile_cells, threads;
    bool use_graph;
    void *stream;                    // cudaStream_t or nullptr
    // bonded records in CSR by bead id: both ends hold the record
    std::vector<int32_t> bptr;       // [n+1]
    std::vector<int32_t> bpartner;   // [2*nbonds]
    std::vector<int32_t> bkind;      // [2*nbonds]
    std::vector<double> br0, bk, balpha;
    int64_t nbonds;
    // cell geometry: n_c = floor(L), h = L / n_c, inv_h = n_c / L
    int32_t nc[3];
    double h[3], inv_h[3];
};

class EngineBase {
  public:
    virtual ~EngineBase() {}
    virtual int set_state(const double *pos, const double *vel, int64_t step) = 0;
    virtual int step(int64_t nsteps) = 0;
    virtual int get_state(double *pos, double *vel, double *force, int64_t *step) = 0;
    virtual int observables(dpd_obs *out) = 0;
    virtual int gr(double rmax, int32_t nbins, uint64_t *counts) = 0;
    virtual int get_cells(uint32_t *key_by_id, int64_t *order, int64_t *cell_start) = 0;
    virtual int sync() = 0;
    virtual int64_t launches() const = 0;
    virtual int profile_begin(int64_t max_steps) = 0;
    virtual int profile_end(double ms[3], int64_t *nsteps) = 0;
    const char *last_error() const { return err_.c_str(); }

  protected:
    std::string err_;
};

// Returns nullptr and sets *rc on failure.
EngineBase *make_engine_f32(const Config &cfg, int *rc, std::string *err);
EngineBase *make_engine_f64(const Config &cfg, int *rc, std::string *err);

}  // namespace dpd
