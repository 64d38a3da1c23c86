// Per-precision engine: owns the device state of one DPD system and
// sequences the kernels of kernels.cuh (Fig. 1 of arxiv 1804.06205).
#pragma once

#include <algorithm>
#include <memory>

#include "kernels.cuh"

namespace dpd {

#define DPD_CU(call)                                                              \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            err_ = std::string(#call) + ": " + cudaGetErrorString(e_);            \
            return DPD_ECUDA;                                                     \
        }                                                                         \
    } while (0)

template <class P>
class Engine : public EngineBase {
    using real = typename P::real;
    using vec4 = typename P::vec4;

    struct GraphSlot {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t ev_node[4] = {nullptr, nullptr, nullptr, nullptr};
        bool timed = false;
        int64_t nkernels = 0;
    };

  public:
    explicit Engine(const Config &c) : cfg_(c) {}

    ~Engine() override {
        if (stream_) cudaStreamSynchronize(stream_);
        for (auto &row : graphs_)
            for (auto &g : row) {
                if (g.exec) cudaGraphExecDestroy(g.exec);
                if (g.graph) cudaGraphDestroy(g.graph);
            }
        for (cudaEvent_t e : prof_ev_) cudaEventDestroy(e);
        for (cudaEvent_t e : ph_)
            if (e) cudaEventDestroy(e);
        for (void *p : allocs_) cudaFree(p);
        if (io_host_) cudaFreeHost(io_host_);
        if (own_stream_ && stream_) cudaStreamDestroy(stream_);
    }

    int init() {
        n_ = (int)cfg_.n;
        geo_.nx = cfg_.nc[0];
        geo_.ny = cfg_.nc[1];
        geo_.nz = cfg_.nc[2];
        geo_.ncell = geo_.nx * geo_.ny * geo_.nz;
        for (int k = 0; k < 3; ++k) {
            geo_.L[k] = cfg_.L[k];
            geo_.h[k] = cfg_.h[k];
            geo_.inv_h[k] = cfg_.inv_h[k];
        }
        if (cfg_.stream) {
            stream_ = (cudaStream_t)cfg_.stream;
        } else {
            DPD_CU(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
            own_stream_ = true;
        }
        const size_t N = (size_t)n_, C = (size_t)geo_.ncell;
        int rc;
        if ((rc = alloc(&pos_, N)) || (rc = alloc(&pos_tmp_, N)) || (rc = alloc(&vel_[0], N)) ||
            (rc = alloc(&vel_[1], N)) || (rc = alloc(&frc_[0], N)) || (rc = alloc(&frc_[1], N)) ||
            (rc = alloc(&vt_, N)) || (rc = alloc(&fpair_, N)) || (rc = alloc(&ev_, N)) ||
            (rc = alloc(&key_, N)) || (rc = alloc(&key_tmp_, N)) || (rc = alloc(&rank_, N)) ||
            (rc = alloc(&src_, N)) || (rc = alloc(&sid_, N)) || (rc = alloc(&id_[0], N)) ||
            (rc = alloc(&id_[1], N)) || (rc = alloc(&inv_perm_, N)) ||
            (rc = alloc(&count_, C)) || (rc = alloc(&cell_start_, C + 1)) ||
            (rc = alloc(&bsum_, C / SCAN_B + 2)) || (rc = alloc(&counter_, 1)) ||
            (rc = alloc(&status_, 1)) || (rc = alloc(&partial_, RED_BLOCKS * RED_K)) ||
            (rc = alloc(&obs_, RED_K)) || (rc = alloc(&acc_, 4)) ||
            (rc = alloc(&io_, 9 * N)) || (rc = alloc(&types_, N)) ||
            (rc = alloc(&a_, (size_t)cfg_.ntypes * cfg_.ntypes)) ||
            (rc = alloc(&bptr_, N + 1)) || (rc = alloc(&bpartner_, cfg_.bpartner.size() + 1)) ||
            (rc = alloc(&bpar_, cfg_.bpartner.size() + 1)))
            return rc;
        for (auto &e : ph_) DPD_CU(cudaEventCreate(&e));
        DPD_CU(cudaMemsetAsync(count_, 0, C * sizeof(uint32_t), stream_));
        DPD_CU(cudaMemsetAsync(status_, 0, sizeof(int), stream_));
        DPD_CU(cudaMemsetAsync(acc_, 0, 4 * sizeof(double), stream_));
        DPD_CU(cudaMemsetAsync(ev_, 0, N * sizeof(vec4), stream_));
        DPD_CU(cudaMemcpyAsync(types_, cfg_.types.data(), N * sizeof(int32_t),
                               cudaMemcpyHostToDevice, stream_));
        std::vector<real> a(cfg_.a.begin(), cfg_.a.end());
        DPD_CU(cudaMemcpyAsync(a_, a.data(), a.size() * sizeof(real), cudaMemcpyHostToDevice,
                               stream_));
        DPD_CU(cudaMemcpyAsync(bptr_, cfg_.bptr.data(), (N + 1) * sizeof(int32_t),
                               cudaMemcpyHostToDevice, stream_));
        const size_t nb = cfg_.bpartner.size();
        if (nb) {
            std::vector<vec4> bp(nb);
            for (size_t b = 0; b < nb; ++b) {
                bp[b].x = (real)cfg_.br0[b];
                bp[b].y = (real)cfg_.bk[b];
                bp[b].z = (real)cfg_.balpha[b];
                bp[b].w = (real)cfg_.bkind[b];
            }
            DPD_CU(cudaMemcpyAsync(bpartner_, cfg_.bpartner.data(), nb * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, stream_));
            DPD_CU(cudaMemcpyAsync(bpar_, bp.data(), nb * sizeof(vec4), cudaMemcpyHostToDevice,
                                   stream_));
        }
        DPD_CU(cudaStreamSynchronize(stream_));
        choose_tiles();
        return set_pair_smem();
    }

    // ---------------------------------------------------------------- state
    int set_state(const double *pos, const double *vel, int64_t step) override {
        int rc = check_status();
        if (rc) return rc;
        const size_t N = (size_t)n_;
        DPD_CU(cudaMemcpyAsync(io_, pos, 3 * N * sizeof(double), cudaMemcpyHostToDevice, stream_));
        DPD_CU(cudaMemcpyAsync(io_ + 3 * N, vel, 3 * N * sizeof(double), cudaMemcpyHostToDevice,
                               stream_));
        InitArgs<P> ia;
        ia.n = n_;
        ia.g = geo_;
        ia.pos_in = io_;
        ia.vel_in = io_ + 3 * N;
        ia.types = types_;
        ia.pos_tmp = pos_tmp_;
        ia.vel = vel_[cur_];      // "old" order = bead-id order
        ia.frc = frc_[cur_];
        ia.key_tmp = key_tmp_;
        ia.rank = rank_;
        ia.count = count_;
        ia.id = id_[cur_];
        ia.status = status_;
        k_init<P><<<blocks(n_), 256, 0, stream_>>>(ia);
        ++launches_;
        DPD_CU(cudaGetLastError());
        host_step_ = step;
        long long s = (long long)step;
        DPD_CU(cudaMemcpyAsync(counter_, &s, sizeof(long long), cudaMemcpyHostToDevice, stream_));
        rc = enqueue_sort();
        if (rc) return rc;
        if ((rc = launch_pair(true)) || (rc = enqueue_bonds(true, true, false))) return rc;
        DPD_CU(cudaStreamSynchronize(stream_));
        int st = 0;
        DPD_CU(cudaMemcpy(&st, status_, sizeof(int), cudaMemcpyDeviceToHost));
        if (st & ST_BADINPUT) {
            st &= ~ST_BADINPUT;
            DPD_CU(cudaMemcpy(status_, &st, sizeof(int), cudaMemcpyHostToDevice));
            has_state_ = false;
            err_ = "non-finite position or velocity";
            return DPD_EINVAL;
        }
        has_state_ = true;
        return check_status();
    }

    int step(int64_t nsteps) override {
        if (!has_state_) return DPD_ENOSTATE;
        if (nsteps < 0) return DPD_EINVAL;
        int rc = peek_status();
        if (rc) return rc;
        for (int64_t k = 0; k < nsteps; ++k) {
            const int64_t s = host_step_ + 1;
            const bool acc = cfg_.sample_every > 0 && (s % cfg_.sample_every) == 0;
            const bool sample = acc || (k == nsteps - 1);
            const int variant = acc ? 2 : (sample ? 1 : 0);
            if (cfg_.use_graph) {
                rc = launch_graph(variant);
            } else {
                rc = enqueue_step(sample, acc);
            }
            if (rc) return rc;
            host_step_ = s;
        }
        return DPD_OK;
    }

    int get_state(double *pos, double *vel, double *force, int64_t *step) override {
        if (!has_state_) return DPD_ENOSTATE;
        const size_t N = (size_t)n_;
        k_unpermute<P><<<blocks(n_), 256, 0, stream_>>>(n_, geo_, pos_, key_, vel_[cur_],
                                                        frc_[cur_], id_[cur_], io_, io_ + 3 * N,
                                                        io_ + 6 * N);
        ++launches_;
        DPD_CU(cudaGetLastError());
        if (pos)
            DPD_CU(cudaMemcpyAsync(pos, io_, 3 * N * sizeof(double), cudaMemcpyDeviceToHost,
                                   stream_));
        if (vel)
            DPD_CU(cudaMemcpyAsync(vel, io_ + 3 * N, 3 * N * sizeof(double),
                                   cudaMemcpyDeviceToHost, stream_));
        if (force)
            DPD_CU(cudaMemcpyAsync(force, io_ + 6 * N, 3 * N * sizeof(double),
                                   cudaMemcpyDeviceToHost, stream_));
        DPD_CU(cudaStreamSynchronize(stream_));
        if (step) *step = host_step_;
        return check_status();
    }

    int observables(dpd_obs *out) override {
        if (!has_state_) return DPD_ENOSTATE;
        double o[RED_K], acc[4];
        DPD_CU(cudaMemcpyAsync(o, obs_, sizeof(o), cudaMemcpyDeviceToHost, stream_));
        DPD_CU(cudaMemcpyAsync(acc, acc_, sizeof(acc), cudaMemcpyDeviceToHost, stream_));
        DPD_CU(cudaStreamSynchronize(stream_));
        std::memset(out, 0, sizeof(*out));
        const double V = geo_.L[0] * geo_.L[1] * geo_.L[2];
        out->step = host_step_;
        out->momentum[0] = o[0];
        out->momentum[1] = o[1];
        out->momentum[2] = o[2];
        out->sum_v2 = o[3];
        out->kT = n_ > 1 ? o[3] / (3.0 * n_ - 3.0) : 0.0;
        out->p_ideal = o[3] / (3.0 * V);
        out->p_cons = o[4] / (3.0 * V);
        out->p_bond = o[6] / (3.0 * V);
        out->p_total = out->p_ideal + out->p_cons + out->p_bond;
        out->e_pair = o[5];
        out->e_bond = o[7];
        out->n_samples = (int64_t)acc[2];
        out->kT_mean = acc[2] > 0 ? acc[0] / acc[2] : 0.0;
        out->p_mean = acc[2] > 0 ? acc[1] / acc[2] : 0.0;
        out->status = check_status();
        return out->status;
    }

    int gr(double rmax, int32_t nbins, uint64_t *counts) override {
        if (!has_state_) return DPD_ENOSTATE;
        if (!(rmax > 0) || nbins <= 0 || nbins > 4096 || !counts) return DPD_EINVAL;
        int K[3];
        for (int k = 0; k < 3; ++k) {
            K[k] = (int)std::ceil(rmax * geo_.inv_h[k]);
            const int nck = k == 0 ? geo_.nx : (k == 1 ? geo_.ny : geo_.nz);
            if (2 * K[k] + 1 > nck) {
                err_ = "dpd_gr: rmax too large for the cell grid";
                return DPD_EINVAL;
            }
        }
        unsigned long long *d = nullptr;
        DPD_CU(cudaMallocAsync((void **)&d, nbins * sizeof(unsigned long long), stream_));
        DPD_CU(cudaMemsetAsync(d, 0, nbins * sizeof(unsigned long long), stream_));
        const double dr = rmax / (double)nbins;
        k_gr<P><<<blocks(n_), 256, nbins * sizeof(unsigned long long), stream_>>>(
            n_, geo_, K[0], K[1], K[2], pos_, key_, cell_start_, rmax, dr, nbins, d);
        ++launches_;
        DPD_CU(cudaGetLastError());
        DPD_CU(cudaMemcpyAsync(counts, d, nbins * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, stream_));
        DPD_CU(cudaFreeAsync(d, stream_));
        DPD_CU(cudaStreamSynchronize(stream_));
        return check_status();
    }

    int get_cells(uint32_t *key_by_id, int64_t *order, int64_t *cell_start) override {
        if (!has_state_) return DPD_ENOSTATE;
        const size_t N = (size_t)n_, C = (size_t)geo_.ncell;
        uint32_t *dk = reinterpret_cast<uint32_t *>(io_);
        int64_t *dord = reinterpret_cast<int64_t *>(io_ + 3 * N);
        k_cells_out<<<blocks(n_), 256, 0, stream_>>>(n_, key_, id_[cur_], dk, dord);
        ++launches_;
        DPD_CU(cudaGetLastError());
        if (key_by_id)
            DPD_CU(cudaMemcpyAsync(key_by_id, dk, N * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                   stream_));
        if (order)
            DPD_CU(cudaMemcpyAsync(order, dord, N * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                   stream_));
        std::vector<uint32_t> cs;
        if (cell_start) {
            cs.resize(C + 1);
            DPD_CU(cudaMemcpyAsync(cs.data(), cell_start_, (C + 1) * sizeof(uint32_t),
                                   cudaMemcpyDeviceToHost, stream_));
        }
        DPD_CU(cudaStreamSynchronize(stream_));
        if (cell_start)
            for (size_t c = 0; c <= C; ++c) cell_start[c] = cs[c];
        return check_status();
    }

    int sync() override {
        DPD_CU(cudaStreamSynchronize(stream_));
        return check_status();
    }

    int64_t launches() const override { return launches_; }

    int profile_begin(int64_t max_steps) override {
        int rc = profile_release();
        if (rc) return rc;
        prof_ev_.assign((size_t)max_steps * 4, nullptr);
        for (auto &e : prof_ev_) DPD_CU(cudaEventCreate(&e));
        prof_max_ = max_steps;
        prof_n_ = 0;
        prof_on_ = true;
        return DPD_OK;
    }

    int profile_end(double ms[3], int64_t *nsteps) override {
        DPD_CU(cudaStreamSynchronize(stream_));
        ms[0] = ms[1] = ms[2] = 0.0;
        for (int64_t i = 0; i < prof_n_; ++i) {
            for (int k = 0; k < 3; ++k) {
                float t = 0.f;
                DPD_CU(cudaEventElapsedTime(&t, prof_ev_[4 * i + k], prof_ev_[4 * i + k + 1]));
                ms[k] += t;
            }
        }
        if (nsteps) *nsteps = prof_n_;
        return profile_release();
    }

  private:
    // ---------------------------------------------------------------- helpers
    template <class T>
    int alloc(T **p, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (e != cudaSuccess) {
            err_ = std::string("cudaMalloc: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? DPD_ENOMEM : DPD_ECUDA;
        }
        allocs_.push_back(q);
        *p = reinterpret_cast<T *>(q);
        return DPD_OK;
    }

    static int blocks(int n, int t = 256) { return std::max(1, (n + t - 1) / t); }

    // Phase boundary k (0..3) of the step being enqueued: a placeholder event
    // while a graph is captured, a timing event when profiling direct launches.
    int mark(int k, bool capturing) {
        if (capturing) {
            // "external" so that the capture turns it into an event-record node
            DPD_CU(cudaEventRecordWithFlags(ph_[k], stream_, cudaEventRecordExternal));
        } else if (prof_on_ && prof_n_ < prof_max_) {
            DPD_CU(cudaEventRecord(prof_ev_[4 * prof_n_ + k], stream_));
            if (k == 3) ++prof_n_;
        }
        return DPD_OK;
    }

    int point_graph_events(GraphSlot &g, bool timed) {
        for (int k = 0; k < 4; ++k) {
            if (!g.ev_node[k]) continue;
            cudaEvent_t e = timed ? prof_ev_[4 * prof_n_ + k] : ph_[k];
            if (!timed && !g.timed) continue;
            DPD_CU(cudaGraphExecEventRecordNodeSetEvent(g.exec, g.ev_node[k], e));
        }
        g.timed = timed;
        return DPD_OK;
    }

    int profile_release() {
        if (prof_ev_.empty()) return DPD_OK;
        DPD_CU(cudaStreamSynchronize(stream_));
        for (auto &row : graphs_)
            for (auto &g : row)
                if (g.exec && g.timed) {
                    int rc = point_graph_events(g, false);
                    if (rc) return rc;
                }
        for (cudaEvent_t e : prof_ev_) cudaEventDestroy(e);
        prof_ev_.clear();
        prof_on_ = false;
        prof_max_ = prof_n_ = 0;
        return DPD_OK;
    }

    int peek_status() {
        if (status_host_) return status_host_;
        return DPD_OK;
    }

    int check_status() {
        if (!status_) return DPD_OK;
        int st = 0;
        cudaError_t e = cudaMemcpy(&st, status_, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) {
            err_ = std::string("status read: ") + cudaGetErrorString(e);
            return DPD_ECUDA;
        }
        if (st & ST_TIMEOUT) status_host_ = DPD_ETIMEOUT;
        else if (st & ST_NONFINITE) status_host_ = DPD_EUNSTABLE;
        if (status_host_ == DPD_EUNSTABLE) err_ = "non-finite position, velocity or observable";
        return status_host_;
    }

    void choose_tiles() {
        // threads per block; bricks of X x 2 x 2 cells holding about 0.85 T beads
        T_ = cfg_.threads > 0 ? cfg_.threads : 128;
        if (T_ != 64 && T_ != 128 && T_ != 256) T_ = 128;
        BY_ = std::min(2, geo_.ny);
        BZ_ = std::min(2, geo_.nz);
        const double per_cell = (double)n_ / (double)geo_.ncell;
        int xmax = cfg_.tile_cells > 0
                       ? cfg_.tile_cells
                       : (int)std::floor(0.85 * T_ / (BY_ * BZ_ * std::max(per_cell, 0.25)));
        xmax = std::max(1, std::min(xmax, PAIR_MAXX));
        X_ = xmax;
        if (cfg_.tile_cells <= 0) {   // the length near xmax that wastes the fewest cells
            int best = xmax, waste = 1 << 30;
            for (int x = std::max(1, xmax - 2); x <= std::min(PAIR_MAXX, xmax + 1); ++x) {
                const int w = ((geo_.nx + x - 1) / x) * x - geo_.nx;
                if (w < waste) {
                    waste = w;
                    best = x;
                }
            }
            X_ = best;
        }
        X_ = std::min(X_, geo_.nx);
        nbx_ = (geo_.nx + X_ - 1) / X_;
        nby_ = (geo_.ny + BY_ - 1) / BY_;
        nbz_ = (geo_.nz + BZ_ - 1) / BZ_;
        nseg_ = nbx_ * nby_ * nbz_;
        // staged capacity: the mean of (BY+2)(BZ+2)(X+2) cells plus ~4 sigma;
        // larger neighbourhoods are staged in chunks (slots must fit 11 bits)
        const double mean = (BY_ + 2) * (BZ_ + 2) * (X_ + 2) * per_cell;
        int cap = (int)std::ceil(mean + 4.0 * std::sqrt(mean) + 32.0);
        cap = (cap + 31) / 32 * 32;
        const int cap_max = (int)((96 * 1024) / (2 * sizeof(vec4)));
        cap_ = std::max(64, std::min(cap, std::min(cap_max, 2016)));
        smem_ = PairSmem<P>::bytes(cap_, X_, T_);
    }

    // dynamic shared memory above the 48 KB default, set once (not while a
    // graph is being captured)
    // (the attribute is per kernel, shared by all handles: only ever raised)
    template <int T, bool S>
    int set_pair_smem_t() {
        if (smem_ <= 48 * 1024) return DPD_OK;
        cudaFuncAttributes fa;
        DPD_CU(cudaFuncGetAttributes(&fa, k_pair<P, T, S>));
        if ((size_t)fa.maxDynamicSharedSizeBytes >= smem_) return DPD_OK;
        DPD_CU(cudaFuncSetAttribute(k_pair<P, T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem_));
        return DPD_OK;
    }

    int set_pair_smem() {
        int rc;
        switch (T_) {
            case 64:
                if ((rc = set_pair_smem_t<64, true>())) return rc;
                return set_pair_smem_t<64, false>();
            case 256:
                if ((rc = set_pair_smem_t<256, true>())) return rc;
                return set_pair_smem_t<256, false>();
            default:
                if ((rc = set_pair_smem_t<128, true>())) return rc;
                return set_pair_smem_t<128, false>();
        }
    }

    template <int T, bool S>
    int launch_pair_t(const PairArgs<P> &pa) {
        k_pair<P, T, S><<<nseg_, T, smem_, stream_>>>(pa);
        ++launches_;
        DPD_CU(cudaGetLastError());
        return DPD_OK;
    }

    int launch_pair(bool sample) {
        PairArgs<P> pa;
        pa.pos = pos_;
        pa.vt = vt_;
        pa.key = key_;
        pa.cell_start = cell_start_;
        pa.fpair = fpair_;
        pa.ev = ev_;
        pa.a = a_;
        pa.ntypes = cfg_.ntypes;
        pa.nx = geo_.nx;
        pa.ny = geo_.ny;
        pa.nz = geo_.nz;
        pa.X = X_;
        pa.BY = BY_;
        pa.BZ = BZ_;
        pa.nbx = nbx_;
        pa.nby = nby_;
        for (int k = 0; k < 3; ++k) pa.h[k] = (real)geo_.h[k];
        pa.gamma = (real)cfg_.gamma;
        pa.sig_sqdt = (real)(std::sqrt(2.0 * cfg_.gamma * cfg_.kT) / std::sqrt(cfg_.dt));
        {   // Philox round keys: (k0, k1) + r (0x9E3779B9, 0xBB67AE85)
            uint32_t k0 = (uint32_t)(cfg_.seed & 0xffffffffull), k1 = (uint32_t)(cfg_.seed >> 32);
            for (int r = 0; r < 10; ++r) {
                pa.rk[2 * r] = k0;
                pa.rk[2 * r + 1] = k1;
                k0 += 0x9E3779B9u;
                k1 += 0xBB67AE85u;
            }
        }
        pa.noise = cfg_.noise;
        pa.counter = counter_;
        pa.cap = cap_;
        switch (T_) {
            case 64: return sample ? launch_pair_t<64, true>(pa) : launch_pair_t<64, false>(pa);
            case 256: return sample ? launch_pair_t<256, true>(pa) : launch_pair_t<256, false>(pa);
            default: return sample ? launch_pair_t<128, true>(pa) : launch_pair_t<128, false>(pa);
        }
    }

    int enqueue_sort() {
        const int C = geo_.ncell;
        const int nb = (C + SCAN_B - 1) / SCAN_B;
        k_scan1<<<nb, SCAN_T, 0, stream_>>>(count_, C, bsum_);
        k_scan2<<<1, SCAN_T, 0, stream_>>>(bsum_, nb, cell_start_, C);
        k_scan3<<<nb, SCAN_T, 0, stream_>>>(count_, C, bsum_, cell_start_);
        k_scatter<<<blocks(n_), 256, 0, stream_>>>(n_, key_tmp_, rank_, cell_start_, id_[cur_],
                                                   src_, sid_);
        k_cellfix<<<blocks(C), 256, 0, stream_>>>(C, cell_start_, src_, sid_);
        const int nxt = cur_ ^ 1;
        GatherArgs<P> ga;
        ga.n = n_;
        ga.lam_dt = (real)(cfg_.lambda * cfg_.dt);
        ga.src = src_;
        ga.sid = sid_;
        ga.pos_tmp = pos_tmp_;
        ga.vel_old = vel_[cur_];
        ga.frc_old = frc_[cur_];
        ga.key_tmp = key_tmp_;
        ga.pos = pos_;
        ga.vel = vel_[nxt];
        ga.frc = frc_[nxt];
        ga.vt = vt_;
        ga.key = key_;
        ga.id = id_[nxt];
        ga.inv_perm = inv_perm_;
        k_gather<P><<<blocks(n_), 256, 0, stream_>>>(ga);
        launches_ += 6;
        cur_ = nxt;
        DPD_CU(cudaGetLastError());
        return DPD_OK;
    }

    // bonds (+ velocity update unless init) (+ reductions if sampled)
    int enqueue_bonds(bool init, bool sample, bool accumulate) {
        BondArgs<P> ba;
        ba.n = n_;
        ba.g = geo_;
        for (int k = 0; k < 3; ++k) {
            ba.L[k] = (real)geo_.L[k];
            ba.h[k] = (real)geo_.h[k];
        }
        ba.half_dt = (real)(0.5 * cfg_.dt);
        ba.fpair = fpair_;
        ba.pos = pos_;
        ba.key = key_;
        ba.id = id_[cur_];
        ba.inv_perm = inv_perm_;
        ba.bptr = bptr_;
        ba.bpartner = bpartner_;
        ba.bpar = bpar_;
        ba.vel = vel_[cur_];
        ba.frc = frc_[cur_];
        ba.ev = ev_;
        if (init) {
            if (sample) k_bond_vel<P, true, true><<<blocks(n_), 256, 0, stream_>>>(ba);
            else k_bond_vel<P, true, false><<<blocks(n_), 256, 0, stream_>>>(ba);
        } else {
            if (sample) k_bond_vel<P, false, true><<<blocks(n_), 256, 0, stream_>>>(ba);
            else k_bond_vel<P, false, false><<<blocks(n_), 256, 0, stream_>>>(ba);
        }
        ++launches_;
        DPD_CU(cudaGetLastError());
        if (sample) {
            k_reduce<P><<<RED_BLOCKS, RED_T, 0, stream_>>>(n_, vel_[cur_], ev_, partial_);
            const double V = geo_.L[0] * geo_.L[1] * geo_.L[2];
            k_reduce_final<<<1, 32, 0, stream_>>>(RED_BLOCKS, partial_, obs_, acc_,
                                                  accumulate ? 1 : 0,
                                                  n_ > 1 ? 1.0 / (3.0 * n_ - 3.0) : 0.0,
                                                  1.0 / (3.0 * V), status_);
            launches_ += 2;
            DPD_CU(cudaGetLastError());
        }
        return DPD_OK;
    }

    int enqueue_step(bool sample, bool accumulate, bool capturing = false) {
        int rc = mark(0, capturing);
        if (rc) return rc;
        UpdArgs<P> ua;
        ua.n = n_;
        ua.g = geo_;
        ua.dt = (real)cfg_.dt;
        ua.half_dt2 = (real)(0.5 * cfg_.dt * cfg_.dt);
        for (int k = 0; k < 3; ++k) {
            ua.hf[k] = (float)geo_.h[k];
            ua.inv_hf[k] = (float)geo_.inv_h[k];
        }
        ua.key = key_;
        ua.pos = pos_;
        ua.vel = vel_[cur_];
        ua.frc = frc_[cur_];
        ua.pos_tmp = pos_tmp_;
        ua.key_tmp = key_tmp_;
        ua.rank = rank_;
        ua.count = count_;
        ua.counter = counter_;
        ua.status = status_;
        k_update<P><<<blocks(n_), 256, 0, stream_>>>(ua);
        ++launches_;
        DPD_CU(cudaGetLastError());
        if ((rc = enqueue_sort()) || (rc = mark(1, capturing)) || (rc = launch_pair(sample)) ||
            (rc = mark(2, capturing)) || (rc = enqueue_bonds(false, sample, accumulate)))
            return rc;
        return mark(3, capturing);
    }


    // One captured step per (parity, variant): the ping-pong buffers swap
    // every step, so a graph is valid for the parity it was captured at.
    int launch_graph(int variant) {
        GraphSlot &g = graphs_[cur_][variant];
        if (!g.exec) {
            const int cur0 = cur_;
            const int64_t l0 = launches_;
            cudaGraph_t graph = nullptr;
            DPD_CU(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
            int rc = enqueue_step(variant >= 1, variant == 2, true);
            cudaError_t e = cudaStreamEndCapture(stream_, &graph);
            if (rc) {
                if (graph) cudaGraphDestroy(graph);
                return rc;
            }
            if (e != cudaSuccess) {
                err_ = std::string("graph capture: ") + cudaGetErrorString(e);
                return DPD_ECUDA;
            }
            e = cudaGraphInstantiate(&g.exec, graph, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(graph);
                err_ = std::string("graph instantiate: ") + cudaGetErrorString(e);
                g.exec = nullptr;
                return DPD_ECUDA;
            }
            g.graph = graph;   // kept: its event-record nodes are retargeted per launch
            size_t nn = 0;
            DPD_CU(cudaGraphGetNodes(graph, nullptr, &nn));
            std::vector<cudaGraphNode_t> nodes(nn);
            DPD_CU(cudaGraphGetNodes(graph, nodes.data(), &nn));
            for (cudaGraphNode_t nd : nodes) {
                cudaGraphNodeType ty;
                DPD_CU(cudaGraphNodeGetType(nd, &ty));
                if (ty != cudaGraphNodeTypeEventRecord) continue;
                cudaEvent_t ev = nullptr;
                DPD_CU(cudaGraphEventRecordNodeGetEvent(nd, &ev));
                for (int k = 0; k < 4; ++k)
                    if (ev == ph_[k]) g.ev_node[k] = nd;
            }
            g.nkernels = launches_ - l0;
            launches_ = l0;
            cur_ = cur0;   // capture did not execute anything
        }
        const bool timed = prof_on_ && prof_n_ < prof_max_;
        if (timed || g.timed) {
            int rc = point_graph_events(g, timed);
            if (rc) return rc;
        }
        DPD_CU(cudaGraphLaunch(g.exec, stream_));
        if (timed) ++prof_n_;
        launches_ += g.nkernels;
        cur_ ^= 1;
        return DPD_OK;
    }

    Config cfg_;
    Geo geo_{};
    int n_ = 0;
    cudaStream_t stream_ = nullptr;
    bool own_stream_ = false;
    std::vector<void *> allocs_;
    vec4 *pos_ = nullptr, *pos_tmp_ = nullptr, *vel_[2] = {nullptr, nullptr},
         *frc_[2] = {nullptr, nullptr}, *vt_ = nullptr, *fpair_ = nullptr, *ev_ = nullptr;
    uint32_t *key_ = nullptr, *key_tmp_ = nullptr, *rank_ = nullptr, *src_ = nullptr;
    int32_t *sid_ = nullptr, *id_[2] = {nullptr, nullptr}, *inv_perm_ = nullptr;
    uint32_t *count_ = nullptr, *cell_start_ = nullptr, *bsum_ = nullptr;
    long long *counter_ = nullptr;
    int *status_ = nullptr;
    double *partial_ = nullptr, *obs_ = nullptr, *acc_ = nullptr, *io_ = nullptr;
    void *io_host_ = nullptr;
    int32_t *types_ = nullptr, *bptr_ = nullptr, *bpartner_ = nullptr;
    vec4 *bpar_ = nullptr;
    real *a_ = nullptr;
    int cur_ = 0;
    bool has_state_ = false;
    int64_t host_step_ = 0;
    int64_t launches_ = 0;
    int status_host_ = 0;
    int T_ = 128, X_ = 1, BY_ = 2, BZ_ = 2, nbx_ = 1, nby_ = 1, nbz_ = 1, nseg_ = 1, cap_ = 256;
    size_t smem_ = 0;
    GraphSlot graphs_[2][3];
    cudaEvent_t ph_[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> prof_ev_;
    int64_t prof_max_ = 0, prof_n_ = 0;
    bool prof_on_ = false;
};

}  // namespace dpd
