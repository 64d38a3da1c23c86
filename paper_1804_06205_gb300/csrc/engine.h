// Host-side interface between the C ABI (dpd_api.cu) and the per-precision
// engines (engine_f32.cu, engine_f64.cu).  No device code here.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "dpd.h"

namespace dpd {

// One system, as dpd_create / dpd_batch_add validated it.
struct Config {
    double L[3];
    int64_t n;
    int32_t ntypes;
    std::vector<int32_t> types;      // [n]
    std::vector<double> a;           // [ntypes*ntypes]
    double gamma, kT, dt, lambda;
    uint64_t seed;
    int32_t noise;
    int32_t tile_cells;              // brick length override (0 = automatic)
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

// Leading bytes of a checkpoint; the records follow in bead-id order.
struct CkptHeader {
    char magic[8];          // "DPDCKPT1"
    uint32_t version;       // 1
    int32_t precision;      // DPD_FP32 / DPD_FP64
    int64_t n, step;        // beads, evaluation counter of the stored force
    int32_t nc[3];          // cells per edge
    uint32_t record_bytes;  // 40 (FP32) or 72 (FP64)
    double L[3];            // box
    uint64_t seed;          // Philox key
};
static_assert(sizeof(CkptHeader) == 80, "checkpoint header layout");

// The pools of a batch and the engine-wide options.
struct BatchConfig {
    int64_t max_beads, max_cells, max_bonds;   // bond records count both ends
    int32_t max_systems;
    int32_t threads;                 // pair-kernel threads per block (0 = auto)
    int32_t sample_every;            // running means every k steps (0 = off)
    bool use_graph;
    bool persistent;                 // one cooperative launch per dpd_step call
    void *stream;                    // cudaStream_t or nullptr
};

class BatchBase {
  public:
    virtual ~BatchBase() {}
    // Reserve space for a system and its parameters; *slot names it.
    virtual int add_system(const Config &cfg, int *slot) = 0;
    virtual int remove_system(int slot) = 0;
    virtual int set_state(int slot, const double *pos, const double *vel, int64_t step) = 0;
    // Advance every resident system (all must have a state).
    virtual int step(int64_t nsteps) = 0;
    virtual int get_state(int slot, double *pos, double *vel, double *force, int64_t *step) = 0;
    virtual int observables(int slot, dpd_obs *out) = 0;
    virtual int gr(int slot, double rmax, int32_t nbins, uint64_t *counts) = 0;
    virtual int get_cells(int slot, uint32_t *key_by_id, int64_t *order, int64_t *cell_start) = 0;
    // Checkpoint of one system: header + per-bead records (CkptHeader below).
    virtual int64_t checkpoint_bytes(int slot) const = 0;
    virtual int get_checkpoint(int slot, void *buf, int64_t bytes) = 0;
    virtual int set_checkpoint(int slot, const void *buf, int64_t bytes) = 0;
    virtual int sync() = 0;
    virtual int64_t launches() const = 0;
    virtual int profile_begin(int64_t max_steps) = 0;
    virtual int profile_end(double ms[3], int64_t *nsteps) = 0;
    // used[4] / cap[4]: beads, cells, bricks, bond records
    virtual void usage(int64_t used[4], int64_t cap[4]) const = 0;
    virtual int nlive() const = 0;
    const char *last_error() const { return err_.c_str(); }

  protected:
    std::string err_;
};

// Returns nullptr and sets *rc / *err on failure.
BatchBase *make_batch_f32(const BatchConfig &bc, int *rc, std::string *err);
BatchBase *make_batch_f64(const BatchConfig &bc, int *rc, std::string *err);

}  // namespace dpd
