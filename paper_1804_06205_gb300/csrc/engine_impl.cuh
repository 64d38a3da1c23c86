// Per-precision batch engine: owns the device pools of any number of
// resident DPD systems and sequences the kernels of kernels.cuh (Fig. 1 of
// arxiv 1804.06205) over all of them.  A single system is a batch of one.
//
// Pools.  Systems are packed one after another, in the same order, in every
// pool: beads [bead0, bead0+n), cells [cell0, cell0+ncell), pair-kernel
// bricks [brick0, ...), bond records [bond0, ...).  Adding a system appends
// it; removing one re-packs the survivors (k_relayout) between steps.
#pragma once

#include <algorithm>
#include <cmath>
#include <memory>

#include "kernels.cuh"
#include "persist.cuh"

namespace dpd {

#define DPD_CU(call)                                                              \
    do {                                                                          \
        cudaError_t e_ = (call);                                                  \
        if (e_ != cudaSuccess) {                                                  \
            err_ = std::string(#call) + ": " + cudaGetErrorString(e_);            \
            return DPD_ECUDA;                                                     \
        }                                                                         \
    } while (0)

static __global__ void k_fill_int(int *p, int n, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}


// Launch with programmatic stream serialization: the kernel may be scheduled
// while the previous kernel of the stream drains, and it waits (griddep_wait,
// its first statement) until that kernel has completed before it touches
// memory.  Used for the kernels of a step, which follow one another.
template <class... KA, class... AA>
static cudaError_t launch_pdl(void (*k)(KA...), int grid, int block, size_t smem, cudaStream_t st,
                              AA &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, std::forward<AA>(args)...);
}

template <class P>
class BatchEngine : public BatchBase {
    using real = typename P::real;
    using vec4 = typename P::vec4;

    struct SysHost {
        Config cfg;
        bool live = false, has_state = false;
        int n = 0, ncell = 0, nbrick = 0, nbond = 0;
        int bead0 = 0, cell0 = 0, brick0 = 0, bond0 = 0;
        int X = 1, BY = 1, BZ = 1, nbx = 1, nby = 1, nbz = 1, cap = 64;
        int64_t step = 0;
        int red0 = 0, nred = 0, rsys_index = 0;   // reduction chunks, entry in rsys
        bool obs_fresh = false;   // obs_ holds the observables of the current state
        bool unsorted = false;    // restored in bead-id order; no cell order or cell starts yet
    };

    struct GraphSlot {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaGraphNode_t ev_node[4] = {nullptr, nullptr, nullptr, nullptr};
        bool timed = false;
        int64_t nkernels = 0;
    };

  public:
    explicit BatchEngine(const BatchConfig &bc) : bc_(bc) {}

    ~BatchEngine() override {
        if (stream_) cudaStreamSynchronize(stream_);
        drop_graphs();
        for (cudaEvent_t e : prof_ev_) cudaEventDestroy(e);
        for (cudaEvent_t e : ph_)
            if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : xev_)
            if (e) cudaEventDestroy(e);
        if (xfer_) cudaStreamDestroy(xfer_);
        for (void *p : allocs_) cudaFree(p);
        if (own_stream_ && stream_) cudaStreamDestroy(stream_);
    }

    int init() {
        NB_ = (int)bc_.max_beads;
        NC_ = (int)bc_.max_cells;
        NBR_ = NC_;                      // a brick holds at least one cell
        NBD_ = (int)std::max<int64_t>(bc_.max_bonds, 1);
        NS_ = std::max(1, bc_.max_systems);
        NRB_ = NB_ / RED_CHUNK + NS_ + 1;
        T_ = bc_.threads > 0 ? bc_.threads : 128;
        if (T_ != 64 && T_ != 128 && T_ != 256) T_ = 128;
        if (bc_.stream) {
            stream_ = (cudaStream_t)bc_.stream;
        } else {
            DPD_CU(cudaStreamCreateWithFlags(&stream_, cudaStreamNonBlocking));
            own_stream_ = true;
        }
        const size_t N = (size_t)NB_, C = (size_t)NC_;
        int rc;
        if ((rc = alloc(&pos_, N)) || (rc = alloc(&pos_tmp_, N)) || (rc = alloc(&vel_[0], N)) ||
            (rc = alloc(&vel_[1], N)) || (rc = alloc(&frc_[0], N)) || (rc = alloc(&frc_[1], N)) ||
            (rc = alloc(&vt_, N)) || (rc = alloc(&ev_, N)) ||
            (rc = alloc(&key_, N)) || (rc = alloc(&key_tmp_, N)) || (rc = alloc(&rank_, N)) ||
            (rc = alloc(&srcid_, N)) || (rc = alloc(&id_[0], N)) ||
            (rc = alloc(&id_[1], N)) || (rc = alloc(&inv_perm_, N)) || (rc = alloc(&bsys_, N)) ||
            (rc = alloc(&types_, N)) ||
            (rc = alloc(&count_, C)) || (rc = alloc(&cell_start_, C + 1)) ||
            (rc = alloc(&bsum_, C / SCAN_B + 2)) || (rc = alloc(&brick_sys_, (size_t)NBR_)) ||
            (rc = alloc(&sys_, (size_t)NS_)) || (rc = alloc(&counter_, (size_t)NS_)) ||
            (rc = alloc(&status_, 1)) || (rc = alloc(&atab_, (size_t)NS_ * PAIR_MAXT * PAIR_MAXT)) ||
            (rc = alloc(&bptr_, N + 1)) || (rc = alloc(&bpartner_, (size_t)NBD_)) ||
            (rc = alloc(&bpar_, (size_t)NBD_)) || (rc = alloc(&rmap_, (size_t)NRB_)) ||
            (rc = alloc(&rsys_, (size_t)NS_)) || (rc = alloc(&partial_, (size_t)NRB_ * RED_K)) ||
            (rc = alloc(&obs_, (size_t)NS_ * RED_K)) || (rc = alloc(&acc_, (size_t)NS_ * 4)) ||
            (rc = alloc(&old_bead0_, (size_t)NS_)) || (rc = alloc(&bar_, 1)))
            return rc;
        if (!P::kOffsets) {   // FP64 Box-Muller logarithm tables
            if ((rc = alloc(&lntab_, 1))) return rc;
            k_ln_tab<<<1, 128, 0, stream_>>>(lntab_);
            DPD_CU(cudaGetLastError());
        }
        for (auto &e : ph_) DPD_CU(cudaEventCreate(&e));
        for (auto &e : xev_) DPD_CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        DPD_CU(cudaStreamCreateWithFlags(&xfer_, cudaStreamNonBlocking));
        DPD_CU(cudaMemsetAsync(count_, 0, C * sizeof(uint32_t), stream_));
        DPD_CU(cudaMemsetAsync(status_, 0, sizeof(int), stream_));
        DPD_CU(cudaMemsetAsync(acc_, 0, (size_t)NS_ * 4 * sizeof(double), stream_));
        DPD_CU(cudaMemsetAsync(obs_, 0, (size_t)NS_ * RED_K * sizeof(double), stream_));
        DPD_CU(cudaMemsetAsync(ev_, 0, N * sizeof(vec4), stream_));
        DPD_CU(cudaMemsetAsync(bptr_, 0, (N + 1) * sizeof(int32_t), stream_));
        DPD_CU(cudaStreamSynchronize(stream_));
        hs_.resize(NS_);
        hsys_.resize(NS_);
        return DPD_OK;
    }

    // ------------------------------------------------------------ membership
    int add_system(const Config &c, int *slot) override {
        int rc0 = flush_removals();
        if (rc0) return rc0;
        int s = -1;
        for (int k = 0; k < NS_; ++k)
            if (!hs_[k].live) {
                s = k;
                break;
            }
        if (s < 0) {
            err_ = "no free system slot";
            return DPD_ENOMEM;
        }
        SysHost h;
        h.cfg = c;
        h.n = (int)c.n;
        h.ncell = c.nc[0] * c.nc[1] * c.nc[2];
        h.nbond = (int)c.bpartner.size();
        choose_tiles(h);
        if (used_beads_ + h.n > NB_ || used_cells_ + h.ncell > NC_ ||
            used_bricks_ + h.nbrick > NBR_ || used_bonds_ + h.nbond > NBD_) {
            err_ = "the system does not fit in the batch's pools";
            return DPD_ENOMEM;
        }
        h.bead0 = used_beads_;
        h.cell0 = used_cells_;
        h.brick0 = used_bricks_;
        h.bond0 = used_bonds_;
        h.live = true;
        hs_[s] = std::move(h);
        order_.push_back(s);
        int rc = upload_system(s);
        if (rc) {
            hs_[s].live = false;
            order_.pop_back();
            return rc;
        }
        used_beads_ += hs_[s].n;
        used_cells_ += hs_[s].ncell;
        used_bricks_ += hs_[s].nbrick;
        used_bonds_ += hs_[s].nbond;
        if ((rc = rebuild_reduce_maps()) || (rc = update_smem())) return rc;
        drop_graphs();
        *slot = s;
        return DPD_OK;
    }

    // Removal frees the slot at once; the survivors are re-packed (one
    // relayout for any number of removals) before the next step or admission.
    int remove_system(int s) override {
        if (s < 0 || s >= NS_ || !hs_[s].live) return DPD_EINVAL;
        hs_[s].live = false;
        order_.erase(std::find(order_.begin(), order_.end(), s));
        repack_pending_ = true;
        return DPD_OK;
    }

    int flush_removals() {
        if (!repack_pending_) return DPD_OK;
        repack_pending_ = false;
        int rc = check_status();
        if (rc) return rc;
        std::vector<int> old0(NS_, 0);
        for (int k : order_) old0[k] = hs_[k].bead0;
        // re-pack the survivors in order; only systems that moved are uploaded
        used_beads_ = used_cells_ = used_bricks_ = used_bonds_ = 0;
        for (int k : order_) {
            SysHost &h = hs_[k];
            const bool moved = h.bead0 != used_beads_ || h.cell0 != used_cells_ ||
                               h.brick0 != used_bricks_ || h.bond0 != used_bonds_;
            h.bead0 = used_beads_;
            h.cell0 = used_cells_;
            h.brick0 = used_bricks_;
            h.bond0 = used_bonds_;
            used_beads_ += h.n;
            used_cells_ += h.ncell;
            used_bricks_ += h.nbrick;
            used_bonds_ += h.nbond;
            if (moved && (rc = upload_system(k, false))) return rc;
        }
        if ((rc = rebuild_reduce_maps()) || (rc = update_smem())) return rc;
        if (used_beads_ > 0) {
            DPD_CU(cudaMemcpyAsync(old_bead0_, old0.data(), NS_ * sizeof(int),
                                   cudaMemcpyHostToDevice, stream_));
            RelayoutArgs<P> ra;
            ra.n_new = used_beads_;
            ra.bsys_new = bsys_;
            ra.sys_new = sys_;
            ra.old_bead0 = old_bead0_;
            ra.pos = pos_;
            ra.vel = vel_[cur_];
            ra.frc = frc_[cur_];
            ra.key = key_;
            ra.id = id_[cur_];
            ra.pos_out = pos_tmp_;
            ra.vel_out = vel_[cur_ ^ 1];
            ra.frc_out = frc_[cur_ ^ 1];
            ra.key_out = key_tmp_;
            ra.id_out = id_[cur_ ^ 1];
            k_relayout<P><<<blocks(used_beads_), 256, 0, stream_>>>(ra);
            ++launches_;
            DPD_CU(cudaGetLastError());
            std::swap(pos_, pos_tmp_);
            std::swap(key_, key_tmp_);
            cur_ ^= 1;
        }
        DPD_CU(cudaStreamSynchronize(stream_));   // also releases the upload staging
        upload_keep_.clear();
        drop_graphs();
        return DPD_OK;
    }

    // ---------------------------------------------------------------- state
    int set_state(int s, const double *pos, const double *vel, int64_t step) override {
        if (s < 0 || s >= NS_ || !hs_[s].live) return DPD_EINVAL;
        int rc = check_status();
        if (rc) return rc;
        SysHost &h = hs_[s];
        const size_t n = (size_t)h.n;
        if ((rc = ensure_io(n))) return rc;
        // the initial binning writes the "old" buffers; the sort brings the
        // system into the current ones, leaving the other systems untouched
        const int old = cur_ ^ 1;
        InitArgs<P> ia;
        ia.s = s;
        ia.sys = sys_;
        ia.pos_in = io_;
        ia.vel_in = io_ + 3 * n;
        ia.types = types_ + h.bead0;
        ia.pos_tmp = pos_tmp_;
        ia.vel = vel_[old];
        ia.frc = frc_[old];
        ia.key_tmp = key_tmp_;
        ia.rank = rank_;
        ia.count = count_;
        ia.id = id_[old];
        ia.status = status_;
        // host -> device in chunks on the copy stream, each binned as soon as
        // it has arrived; the copies wait for earlier work on io_
        const int nch = io_chunks(h.n);
        DPD_CU(cudaEventRecord(xev_[IO_MAXCH], stream_));
        DPD_CU(cudaStreamWaitEvent(xfer_, xev_[IO_MAXCH], 0));
        for (int c = 0; c < nch; ++c) {
            const size_t i0 = (size_t)h.n * c / nch, i1 = (size_t)h.n * (c + 1) / nch;
            DPD_CU(cudaMemcpyAsync(io_ + 3 * i0, pos + 3 * i0, 3 * (i1 - i0) * sizeof(double),
                                   cudaMemcpyHostToDevice, xfer_));
            DPD_CU(cudaMemcpyAsync(io_ + 3 * n + 3 * i0, vel + 3 * i0,
                                   3 * (i1 - i0) * sizeof(double), cudaMemcpyHostToDevice, xfer_));
            DPD_CU(cudaEventRecord(xev_[c], xfer_));
            DPD_CU(cudaStreamWaitEvent(stream_, xev_[c], 0));
            ia.i0 = (int)i0;
            ia.i1 = (int)i1;
            k_init<P><<<blocks((int)(i1 - i0)), 256, 0, stream_>>>(ia);
            ++launches_;
            DPD_CU(cudaGetLastError());
        }
        long long sv = (long long)step;
        DPD_CU(cudaMemcpyAsync(counter_ + s, &sv, sizeof(long long), cudaMemcpyHostToDevice,
                               stream_));
        if ((rc = enqueue_sort(h.bead0, h.bead0 + h.n, h.cell0, h.cell0 + h.ncell, old, cur_)) ||
            (rc = launch_pair(false, h.brick0, h.nbrick, frc_[cur_])) ||
            (rc = enqueue_bonds(true, false, h.bead0, h.bead0 + h.n)))
            return rc;
        h.unsorted = false;
        h.obs_fresh = false;
        DPD_CU(cudaStreamSynchronize(stream_));
        int st = 0;
        DPD_CU(cudaMemcpy(&st, status_, sizeof(int), cudaMemcpyDeviceToHost));
        if (st & ST_BADINPUT) {
            st &= ~ST_BADINPUT;
            DPD_CU(cudaMemcpy(status_, &st, sizeof(int), cudaMemcpyHostToDevice));
            h.has_state = false;
            err_ = "non-finite position or velocity";
            return DPD_EINVAL;
        }
        h.has_state = true;
        h.step = step;
        return check_status();
    }

    int step(int64_t nsteps) override {
        if (nsteps < 0) return DPD_EINVAL;
        int rc0 = flush_removals();
        if (rc0) return rc0;
        if (order_.empty()) return nsteps == 0 ? DPD_OK : DPD_ENOSTATE;
        for (int k : order_)
            if (!hs_[k].has_state) return DPD_ENOSTATE;
        int rc = peek_status();
        if (rc) return rc;
        if (nsteps > 0 && bc_.persistent && bc_.sample_every == 0 && !bc_.use_graph &&
            persist_grid_ > 0) {
            if ((rc = launch_persistent(nsteps))) return rc;
            for (int s : order_) {
                hs_[s].step += nsteps;
                hs_[s].obs_fresh = false;
                hs_[s].unsorted = false;
            }
            return DPD_OK;
        }
        // Step kinds: 0 plain, its bond kernel also doing the next step's position
        // update (which that step then skips); 1 plain without it, the last step of
        // a call; 2 sampled for the running means.  Observables are otherwise
        // computed on demand from the state (observables()).
        bool updated = false, sampled = false;
        for (int64_t k = 0; k < nsteps; ++k) {
            // running means: one system's steps decide when (a batch of one)
            const bool acc = bc_.sample_every > 0 && order_.size() == 1 &&
                             ((hs_[order_[0]].step + 1) % bc_.sample_every) == 0;
            const int base = acc ? 2 : (k == nsteps - 1 ? 1 : 0);
            const int variant = base + (updated ? 3 : 0);
            rc = bc_.use_graph ? launch_graph(variant)
                               : enqueue_step(acc, acc, false, !updated, base == 0);
            if (rc) return rc;
            updated = base == 0;
            sampled = acc;
            for (int s : order_) hs_[s].step += 1;
        }
        if (nsteps > 0)
            for (int s : order_) {
                hs_[s].obs_fresh = sampled;
                hs_[s].unsorted = false;
            }
        return DPD_OK;
    }

    int get_state(int s, double *pos, double *vel, double *force, int64_t *step) override {
        if (s < 0 || s >= NS_ || !hs_[s].live) return DPD_EINVAL;
        SysHost &h = hs_[s];
        if (!h.has_state) return DPD_ENOSTATE;
        const size_t n = (size_t)h.n;
        int rc = ensure_io(n);
        if (rc) return rc;
        k_inv_perm<<<blocks(h.n), 256, 0, stream_>>>(h.bead0, h.n, id_[cur_], inv_perm_);
        ++launches_;
        DPD_CU(cudaGetLastError());
        // read out in chunks of ids, each copied to the host on the copy stream
        // while the next one is gathered
        const int nch = io_chunks(h.n);
        for (int c = 0; c < nch; ++c) {
            const size_t i0 = (size_t)h.n * c / nch, i1 = (size_t)h.n * (c + 1) / nch;
            k_unpermute<P><<<blocks((int)(i1 - i0)), 256, 0, stream_>>>(
                s, (int)i0, (int)i1, sys_, pos_, key_, vel_[cur_], frc_[cur_], inv_perm_, io_,
                io_ + 3 * n, io_ + 6 * n);
            ++launches_;
            DPD_CU(cudaGetLastError());
            DPD_CU(cudaEventRecord(xev_[c], stream_));
            DPD_CU(cudaStreamWaitEvent(xfer_, xev_[c], 0));
            const size_t b = 3 * (i1 - i0) * sizeof(double);
            if (pos)
                DPD_CU(cudaMemcpyAsync(pos + 3 * i0, io_ + 3 * i0, b, cudaMemcpyDeviceToHost,
                                       xfer_));
            if (vel)
                DPD_CU(cudaMemcpyAsync(vel + 3 * i0, io_ + 3 * n + 3 * i0, b,
                                       cudaMemcpyDeviceToHost, xfer_));
            if (force)
                DPD_CU(cudaMemcpyAsync(force + 3 * i0, io_ + 6 * n + 3 * i0, b,
                                       cudaMemcpyDeviceToHost, xfer_));
        }
        DPD_CU(cudaStreamSynchronize(xfer_));
        DPD_CU(cudaStreamSynchronize(stream_));
        if (step) *step = h.step;
        return check_status();
    }

    int observables(int s, dpd_obs *out) override {
        if (s < 0 || s >= NS_ || !hs_[s].live) return DPD_EINVAL;
        SysHost &h = hs_[s];
        if (!h.has_state) return DPD_ENOSTATE;
        if (!h.obs_fresh) {   // the sampled pair sums and the bond sums of this state
            int rc = check_status();
            if (rc || (rc = ensure_sorted(s))) return rc;
            // the forces go to the other buffer, free between steps; only the
            // sampled sums are kept
            if ((rc = launch_pair(true, h.brick0, h.nbrick, frc_[cur_ ^ 1])) ||
                (h.nbond > 0 && (rc = enqueue_bonds(false, false, h.bead0, h.bead0 + h.n,
                                                    false, true))) ||
                (rc = enqueue_reduce(h.red0, h.nred, h.rsys_index, 1, false)))
                return rc;
            h.obs_fresh = true;
        }
        double o[RED_K], acc[4];
        DPD_CU(cudaMemcpyAsync(o, obs_ + (size_t)s * RED_K, sizeof(o), cudaMemcpyDeviceToHost,
                               stream_));
        DPD_CU(cudaMemcpyAsync(acc, acc_ + (size_t)s * 4, sizeof(acc), cudaMemcpyDeviceToHost,
                               stream_));
        DPD_CU(cudaStreamSynchronize(stream_));
        std::memset(out, 0, sizeof(*out));
        const double V = h.cfg.L[0] * h.cfg.L[1] * h.cfg.L[2];
        out->step = h.step;
        out->momentum[0] = o[0];
        out->momentum[1] = o[1];
        out->momentum[2] = o[2];
        out->sum_v2 = o[3];
        out->kT = h.n > 1 ? o[3] / (3.0 * h.n - 3.0) : 0.0;
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

    int gr(int s, double rmax, int32_t nbins, uint64_t *counts) override {
        if (s < 0 || s >= NS_ || !hs_[s].live) return DPD_EINVAL;
        SysHost &h = hs_[s];
        if (!h.has_state) return DPD_ENOSTATE;
        if (!(rmax > 0) || nbins <= 0 || nbins > 4096 || !counts) return DPD_EINVAL;
        int rc0 = ensure_sorted(s);
        if (rc0) return rc0;
        int K[3];
        for (int k = 0; k < 3; ++k) {
            K[k] = (int)std::ceil(rmax * h.cfg.inv_h[k]);
            if (2 * K[k] + 1 > h.cfg.nc[k]) {
                err_ = "dpd_gr: rmax too large for the cell grid";
                return DPD_EINVAL;
            }
        }
        unsigned long long *d = nullptr;
        DPD_CU(cudaMallocAsync((void **)&d, nbins * sizeof(unsigned long long), stream_));
        DPD_CU(cudaMemsetAsync(d, 0, nbins * sizeof(unsigned long long), stream_));
        const double dr = rmax / (double)nbins;
        k_gr<P><<<blocks(h.n), 256, nbins * sizeof(unsigned long long), stream_>>>(
            s, sys_, K[0], K[1], K[2], pos_, key_, cell_start_, rmax, dr, nbins, d);
        ++launches_;
        DPD_CU(cudaGetLastError());
        DPD_CU(cudaMemcpyAsync(counts, d, nbins * sizeof(unsigned long long),
                               cudaMemcpyDeviceToHost, stream_));
        DPD_CU(cudaFreeAsync(d, stream_));
        DPD_CU(cudaStreamSynchronize(stream_));
        return check_status();
    }

    int get_cells(int s, uint32_t *key_by_id, int64_t *order, int64_t *cell_start) override {
        if (s < 0 || s >= NS_ || !hs_[s].live) return DPD_EINVAL;
        SysHost &h = hs_[s];
        if (!h.has_state) return DPD_ENOSTATE;
        const size_t n = (size_t)h.n, C = (size_t)h.ncell;
        int rc = ensure_io(n);
        if (rc || (rc = ensure_sorted(s))) return rc;
        uint32_t *dk = reinterpret_cast<uint32_t *>(io_);
        int64_t *dord = reinterpret_cast<int64_t *>(io_ + 3 * n);
        k_cells_out<P><<<blocks(h.n), 256, 0, stream_>>>(s, sys_, key_, id_[cur_], dk, dord);
        ++launches_;
        DPD_CU(cudaGetLastError());
        if (key_by_id)
            DPD_CU(cudaMemcpyAsync(key_by_id, dk, n * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                   stream_));
        if (order)
            DPD_CU(cudaMemcpyAsync(order, dord, n * sizeof(int64_t), cudaMemcpyDeviceToHost,
                                   stream_));
        std::vector<uint32_t> cs;
        if (cell_start) {
            cs.resize(C + 1);
            DPD_CU(cudaMemcpyAsync(cs.data(), cell_start_ + h.cell0, (C + 1) * sizeof(uint32_t),
                                   cudaMemcpyDeviceToHost, stream_));
        }
        DPD_CU(cudaStreamSynchronize(stream_));
        if (cell_start)
            for (size_t c = 0; c <= C; ++c) cell_start[c] = (int64_t)cs[c] - h.bead0;
        return check_status();
    }

    // ------------------------------------------------------------ checkpoints
    using Rec = typename CkptRec<P>::type;

    int64_t checkpoint_bytes(int s) const override {
        if (s < 0 || s >= NS_ || !hs_[s].live) return 0;
        return (int64_t)sizeof(CkptHeader) + (int64_t)hs_[s].n * (int64_t)sizeof(Rec);
    }

    int get_checkpoint(int s, void *buf, int64_t bytes) override {
        if (s < 0 || s >= NS_ || !hs_[s].live || !buf) return DPD_EINVAL;
        SysHost &h = hs_[s];
        if (!h.has_state) return DPD_ENOSTATE;
        if (bytes < checkpoint_bytes(s)) {
            err_ = "checkpoint buffer too small (see dpd_checkpoint_bytes)";
            return DPD_EINVAL;
        }
        k_inv_perm<<<blocks(h.n), 256, 0, stream_>>>(h.bead0, h.n, id_[cur_], inv_perm_);
        ++launches_;
        DPD_CU(cudaGetLastError());
        CkptHeader hd;
        fill_header(h, hd);
        // (records stored by the kernel straight into a page-locked host buffer
        // took 0.76 ms at N = 3M, against 0.71 ms for the chunked copies below)
        int rc = ensure_io((size_t)h.n);   // 72 B per bead: holds either record
        if (rc) return rc;
        std::memcpy(buf, &hd, sizeof(hd));
        // records in chunks of ids, each copied to the host on the copy stream
        // while the next one is gathered
        Rec *dst = reinterpret_cast<Rec *>(static_cast<char *>(buf) + sizeof(hd));
        Rec *rio = reinterpret_cast<Rec *>(io_);
        const int nch = io_chunks(h.n);
        for (int c = 0; c < nch; ++c) {
            const int i0 = (int)((int64_t)h.n * c / nch), i1 = (int)((int64_t)h.n * (c + 1) / nch);
            k_ckpt_out<P><<<blocks(i1 - i0), CKPT_BLOCK, 0, stream_>>>(s, i0, i1, sys_, pos_, key_,
                                                                 vel_[cur_], frc_[cur_],
                                                                 inv_perm_, rio);
            ++launches_;
            DPD_CU(cudaGetLastError());
            DPD_CU(cudaEventRecord(xev_[c], stream_));
            DPD_CU(cudaStreamWaitEvent(xfer_, xev_[c], 0));
            DPD_CU(cudaMemcpyAsync(dst + i0, rio + i0, (size_t)(i1 - i0) * sizeof(Rec),
                                   cudaMemcpyDeviceToHost, xfer_));
        }
        DPD_CU(cudaStreamSynchronize(xfer_));
        DPD_CU(cudaStreamSynchronize(stream_));
        return check_status();
    }

    int set_checkpoint(int s, const void *buf, int64_t bytes) override {
        if (s < 0 || s >= NS_ || !hs_[s].live || !buf) return DPD_EINVAL;
        int rc = check_status();
        if (rc) return rc;
        SysHost &h = hs_[s];
        if (bytes < checkpoint_bytes(s)) {
            err_ = "checkpoint too short for this system";
            return DPD_EINVAL;
        }
        CkptHeader want, got;
        fill_header(h, want);
        std::memcpy(&got, buf, sizeof(got));
        if (std::memcmp(got.magic, want.magic, 8) || got.version != want.version ||
            got.precision != want.precision || got.n != want.n ||
            got.record_bytes != want.record_bytes || std::memcmp(got.nc, want.nc, sizeof(got.nc)) ||
            std::memcmp(got.L, want.L, sizeof(got.L)) || got.seed != want.seed) {
            err_ = "checkpoint does not belong to a system of this precision, size, box and seed";
            return DPD_EINVAL;
        }
        const Rec *rec = reinterpret_cast<const Rec *>(static_cast<const char *>(buf) + sizeof(got));
        const char *mh = static_cast<const char *>(mapped_host(buf));
        if (!mh && (rc = ensure_io((size_t)h.n))) return rc;
        // the records go straight into the state arrays, in bead-id order: the
        // next step's position update takes the beads in any order and its cell
        // division puts them in the canonical order, so no sort is spent here;
        // calls that need the cell order first sort (ensure_sorted)
        InitArgs<P> ia;
        ia.s = s;
        ia.sys = sys_;
        ia.pos_in = ia.vel_in = nullptr;
        ia.types = types_ + h.bead0;
        ia.pos_tmp = pos_;
        ia.vel = vel_[cur_];
        ia.frc = frc_[cur_];
        ia.key_tmp = key_;
        ia.rank = nullptr;
        ia.count = nullptr;
        ia.id = id_[cur_];
        ia.status = status_;
        // page-locked host buffer: the kernel reads the records there itself;
        // else they are copied in chunks on the copy stream, each restored as
        // soon as it has landed (the staging buffer is free once earlier work
        // is done)
        Rec *rio = reinterpret_cast<Rec *>(io_);
        const int nch = mh ? 0 : io_chunks(h.n);
        if (mh) {
            ia.i0 = 0;
            ia.i1 = h.n;
            k_ckpt_in<P><<<blocks(h.n), CKPT_BLOCK, 0, stream_>>>(
                ia, reinterpret_cast<const Rec *>(mh + sizeof(got)));
            ++launches_;
            DPD_CU(cudaGetLastError());
        } else {
            DPD_CU(cudaEventRecord(xev_[IO_MAXCH], stream_));
            DPD_CU(cudaStreamWaitEvent(xfer_, xev_[IO_MAXCH], 0));
        }
        for (int c = 0; c < nch; ++c) {
            const int i0 = (int)((int64_t)h.n * c / nch), i1 = (int)((int64_t)h.n * (c + 1) / nch);
            DPD_CU(cudaMemcpyAsync(rio + i0, rec + i0, (size_t)(i1 - i0) * sizeof(Rec),
                                   cudaMemcpyHostToDevice, xfer_));
            DPD_CU(cudaEventRecord(xev_[c], xfer_));
            DPD_CU(cudaStreamWaitEvent(stream_, xev_[c], 0));
            ia.i0 = i0;
            ia.i1 = i1;
            k_ckpt_in<P><<<blocks(i1 - i0), CKPT_BLOCK, 0, stream_>>>(ia, rio);
            ++launches_;
            DPD_CU(cudaGetLastError());
        }
        long long sv = (long long)got.step;
        DPD_CU(cudaMemcpyAsync(counter_ + s, &sv, sizeof(long long), cudaMemcpyHostToDevice,
                               stream_));
        h.unsorted = true;
        h.obs_fresh = false;
        DPD_CU(cudaStreamSynchronize(stream_));
        int st = 0;
        DPD_CU(cudaMemcpy(&st, status_, sizeof(int), cudaMemcpyDeviceToHost));
        if (st & ST_BADINPUT) {
            st &= ~ST_BADINPUT;
            DPD_CU(cudaMemcpy(status_, &st, sizeof(int), cudaMemcpyHostToDevice));
            h.has_state = false;
            err_ = "checkpoint holds a non-finite value or a cell key out of range";
            return DPD_EINVAL;
        }
        h.has_state = true;
        h.step = got.step;
        return check_status();
    }

    // A system restored in bead-id order gets its cell order and cell starts
    // (the cell division of set_state, from the state arrays) before a call
    // that needs them; a step does this by itself.
    int ensure_sorted(int s) {
        SysHost &h = hs_[s];
        if (!h.unsorted) return DPD_OK;
        const int old = cur_ ^ 1;
        k_resort_prep<P><<<blocks(h.n), 256, 0, stream_>>>(
            s, sys_, pos_, key_, vel_[cur_], frc_[cur_], id_[cur_], pos_tmp_, key_tmp_, rank_,
            count_, vel_[old], frc_[old], id_[old]);
        ++launches_;
        DPD_CU(cudaGetLastError());
        int rc = enqueue_sort(h.bead0, h.bead0 + h.n, h.cell0, h.cell0 + h.ncell, old, cur_, true);
        if (rc) return rc;
        h.unsorted = false;
        return DPD_OK;
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

    void usage(int64_t used[4], int64_t cap[4]) const override {
        used[0] = used[1] = used[2] = used[3] = 0;   // the live systems (re-packed or not)
        for (int k : order_) {
            used[0] += hs_[k].n;
            used[1] += hs_[k].ncell;
            used[2] += hs_[k].nbrick;
            used[3] += hs_[k].nbond;
        }
        cap[0] = NB_;
        cap[1] = NC_;
        cap[2] = NBR_;
        cap[3] = NBD_;
    }

    int nlive() const override { return (int)order_.size(); }

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

    void fill_header(const SysHost &h, CkptHeader &hd) const {
        std::memset(&hd, 0, sizeof(hd));
        std::memcpy(hd.magic, "DPDCKPT1", 8);
        hd.version = 1;
        hd.precision = P::kOffsets ? DPD_FP32 : DPD_FP64;
        hd.n = h.n;
        hd.step = h.step;
        for (int k = 0; k < 3; ++k) {
            hd.nc[k] = h.cfg.nc[k];
            hd.L[k] = h.cfg.L[k];
        }
        hd.record_bytes = (uint32_t)sizeof(Rec);
        hd.seed = h.cfg.seed;
    }

    // staging for one system's host <-> device copies (9 doubles per bead)
    // Host-transfer staging for n beads (pos, vel, force as doubles).  Every
    // earlier use has been synchronised, so a smaller buffer is freed at once.
    int ensure_io(size_t n) {
        if (io_n_ >= n) return DPD_OK;
        if (io_) {
            allocs_.erase(std::find(allocs_.begin(), allocs_.end(), (void *)io_));
            cudaFree(io_);
            io_ = nullptr;
            io_n_ = 0;
        }
        double *q = nullptr;
        const int rc = alloc(&q, 9 * n);
        if (rc) return rc;
        io_ = q;
        io_n_ = n;
        return DPD_OK;
    }

    static int blocks(int n, int t = 256) { return std::max(1, (n + t - 1) / t); }

    // the only resident system when there is one (its kernels then need no
    // bead -> system map), else -1
    int sys1() const { return order_.size() == 1 ? order_[0] : -1; }

    // chunks of a host <-> device state transfer: at least IO_CHUNK beads each
    static int io_chunks(int n) { return std::max(1, std::min(IO_MAXCH, n / IO_CHUNK)); }
    // The device address of a caller's buffer that is page-locked host memory
    // mapped into the device's address space (cudaHostAlloc, cudaHostRegister)
    // and 8-byte aligned, so that kernels read or write it over the host link
    // with no copy of their own; null for any other buffer.
    static void *mapped_host(const void *buf) {
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, buf) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        if (at.type != cudaMemoryTypeHost || !at.devicePointer ||
            (reinterpret_cast<uintptr_t>(at.devicePointer) & 7u) != 0)
            return nullptr;
        return at.devicePointer;
    }

    int peek_status() { return status_host_; }

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
        if (status_host_ == DPD_ETIMEOUT) err_ = "a bounded device wait gave up (pair-kernel staging)";
        return status_host_;
    }

    // Brick shape of one system: X x 2 x 2 cells holding about 0.85 T beads,
    // with the length near that which wastes the fewest cells along x.
    void choose_tiles(SysHost &h) const {
        const Config &c = h.cfg;
        h.BY = std::min(2, c.nc[1]);
        h.BZ = std::min(2, c.nc[2]);
        const double per_cell = (double)h.n / (double)h.ncell;
        int xmax = c.tile_cells > 0
                       ? c.tile_cells
                       : (int)std::floor(0.85 * T_ / (h.BY * h.BZ * std::max(per_cell, 0.25)));
        xmax = std::max(1, std::min(xmax, PAIR_MAXX));
        int X = xmax;
        if (c.tile_cells <= 0) {
            int best = xmax, waste = 1 << 30;
            for (int x = std::max(1, xmax - 2); x <= std::min(PAIR_MAXX, xmax + 1); ++x) {
                const int w = ((c.nc[0] + x - 1) / x) * x - c.nc[0];
                if (w < waste) {
                    waste = w;
                    best = x;
                }
            }
            X = best;
        }
        h.X = std::min(X, c.nc[0]);
        h.nbx = (c.nc[0] + h.X - 1) / h.X;
        h.nby = (c.nc[1] + h.BY - 1) / h.BY;
        h.nbz = (c.nc[2] + h.BZ - 1) / h.BZ;
        h.nbrick = h.nbx * h.nby * h.nbz;
        // staged capacity: the mean of (BY+2)(BZ+2)(X+2) cells plus ~4 sigma;
        // larger neighbourhoods are staged in chunks (slots must fit 11 bits)
        const double mean = (h.BY + 2) * (h.BZ + 2) * (h.X + 2) * per_cell;
        int cap = (int)std::ceil(mean + 3.0 * std::sqrt(mean) + 8.0);
        cap = (cap + 15) / 16 * 16;
        const int cap_max = (int)((96 * 1024) / (2 * sizeof(vec4)));
        h.cap = std::max(64, std::min(cap, std::min(cap_max, 2016)));
    }

    // Descriptor, bead -> system and brick -> system maps, a_ij table and
    // bond records of system s at its current place in the pools.
    int upload_system(int s, bool sync = true) {
        SysHost &h = hs_[s];
        const Config &c = h.cfg;
        SysDesc<P> &d = hsys_[s];
        std::memset(&d, 0, sizeof(d));
        d.n = h.n;
        d.bead0 = h.bead0;
        d.cell0 = h.cell0;
        d.ncell = h.ncell;
        d.nx = c.nc[0];
        d.ny = c.nc[1];
        d.nz = c.nc[2];
        d.ntypes = c.ntypes;
        d.brick0 = h.brick0;
        d.X = h.X;
        d.BY = h.BY;
        d.BZ = h.BZ;
        d.nbx = h.nbx;
        d.nby = h.nby;
        d.nbz = h.nbz;
        d.cap = h.cap;
        d.a_off = s * PAIR_MAXT * PAIR_MAXT;
        d.noise = c.noise;
        for (int k = 0; k < 3; ++k) {
            d.L[k] = c.L[k];
            d.h[k] = c.h[k];
            d.inv_h[k] = c.inv_h[k];
            d.hf[k] = (float)c.h[k];
            d.inv_hf[k] = (float)c.inv_h[k];
        }
        d.dt = (real)c.dt;
        d.half_dt2 = (real)(0.5 * c.dt * c.dt);
        d.half_dt = (real)(0.5 * c.dt);
        d.lam_dt = (real)(c.lambda * c.dt);
        d.gamma = (real)c.gamma;
        d.sig_sqdt = (real)(std::sqrt(2.0 * c.gamma * c.kT) / std::sqrt(c.dt));
        {   // Philox round keys: (k0, k1) + r (0x9E3779B9, 0xBB67AE85)
            uint32_t k0 = (uint32_t)(c.seed & 0xffffffffull), k1 = (uint32_t)(c.seed >> 32);
            for (int r = 0; r < 10; ++r) {
                d.rk[2 * r] = k0;
                d.rk[2 * r + 1] = k1;
                k0 += 0x9E3779B9u;
                k1 += 0xBB67AE85u;
            }
        }
        DPD_CU(cudaMemcpyAsync(sys_ + s, &d, sizeof(d), cudaMemcpyHostToDevice, stream_));
        k_fill_int<<<blocks(h.n), 256, 0, stream_>>>(bsys_ + h.bead0, h.n, s);
        k_fill_int<<<blocks(h.nbrick), 256, 0, stream_>>>(brick_sys_ + h.brick0, h.nbrick, s);
        launches_ += 2;
        DPD_CU(cudaGetLastError());
        std::vector<real> a(c.a.begin(), c.a.end());
        DPD_CU(cudaMemcpyAsync(atab_ + d.a_off, a.data(), a.size() * sizeof(real),
                               cudaMemcpyHostToDevice, stream_));
        std::vector<int32_t> bp(c.bptr.begin(), c.bptr.end());
        for (auto &v : bp) v += h.bond0;
        DPD_CU(cudaMemcpyAsync(bptr_ + h.bead0, bp.data(), bp.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, stream_));
        // bead types in id order, resident for every later set_state
        DPD_CU(cudaMemcpyAsync(types_ + h.bead0, c.types.data(), (size_t)h.n * sizeof(int32_t),
                               cudaMemcpyHostToDevice, stream_));
        const size_t nb = c.bpartner.size();
        std::vector<vec4> par(nb);
        if (nb) {
            for (size_t b = 0; b < nb; ++b) {
                par[b].x = (real)c.br0[b];
                par[b].y = (real)c.bk[b];
                par[b].z = (real)c.balpha[b];
                par[b].w = (real)c.bkind[b];
            }
            DPD_CU(cudaMemcpyAsync(bpartner_ + h.bond0, c.bpartner.data(), nb * sizeof(int32_t),
                                   cudaMemcpyHostToDevice, stream_));
            DPD_CU(cudaMemcpyAsync(bpar_ + h.bond0, par.data(), nb * sizeof(vec4),
                                   cudaMemcpyHostToDevice, stream_));
        }
        // the host buffers above must outlive the asynchronous copies: wait now,
        // or keep them until the caller's next synchronisation
        if (sync) {
            DPD_CU(cudaStreamSynchronize(stream_));
        } else {
            upload_keep_.push_back(std::make_shared<UploadBufs>(std::move(a), std::move(bp),
                                                                std::move(par)));
        }
        return DPD_OK;
    }

    // Reduction chunks of every live system, in pool order.
    int rebuild_reduce_maps() {
        std::vector<int2> rmap;
        std::vector<int4> rsys;
        for (int s : order_) {
            SysHost &h = hs_[s];
            h.red0 = (int)rmap.size();
            for (int b = 0; b < h.n; b += RED_CHUNK)
                rmap.push_back(make_int2(h.bead0 + b, h.bead0 + std::min(h.n, b + RED_CHUNK)));
            h.nred = (int)rmap.size() - h.red0;
            h.rsys_index = (int)rsys.size();
            rsys.push_back(make_int4(s, h.red0, h.nred, 0));
        }
        nred_all_ = (int)rmap.size();
        nrsys_all_ = (int)rsys.size();
        if (nred_all_ > NRB_) {
            err_ = "too many reduction chunks";
            return DPD_ENOMEM;
        }
        if (!rmap.empty())
            DPD_CU(cudaMemcpyAsync(rmap_, rmap.data(), rmap.size() * sizeof(int2),
                                   cudaMemcpyHostToDevice, stream_));
        if (!rsys.empty())
            DPD_CU(cudaMemcpyAsync(rsys_, rsys.data(), rsys.size() * sizeof(int4),
                                   cudaMemcpyHostToDevice, stream_));
        DPD_CU(cudaStreamSynchronize(stream_));
        return DPD_OK;
    }

    // shared memory of the pair kernel: the largest brick among live systems
    int update_smem() {
        int capmax = 64, xmax = 1, ntmax = 1;
        for (int s : order_) {
            capmax = std::max(capmax, hs_[s].cap);
            xmax = std::max(xmax, hs_[s].X);
            ntmax = std::max(ntmax, (int)hs_[s].cfg.ntypes);
        }
        if (capmax != capmax_ || xmax != xmax_ || ntmax != ntmax_) drop_graphs();
        capmax_ = capmax;
        xmax_ = xmax;
        ntmax_ = ntmax;
        smem_ = PairSmem<P>::bytes(capmax_, xmax_, T_, ntmax_, true);
        smem_n_ = PairSmem<P>::bytes(capmax_, xmax_, T_, ntmax_, false);
        int rc;
        if (bc_.persistent) {
            switch (T_) {
                case 64: rc = set_persist_t<64>(); break;
                case 256: rc = set_persist_t<256>(); break;
                default: rc = set_persist_t<128>(); break;
            }
            if (rc) return rc;
        }
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

    // (the attribute is per kernel, shared by all handles: only ever raised)
    template <int T, bool S>
    int set_pair_smem_t() {
        const size_t need = S ? smem_ : smem_n_;
        if (need <= 48 * 1024) return DPD_OK;
        cudaFuncAttributes fa;
        DPD_CU(cudaFuncGetAttributes(&fa, k_pair<P, T, S>));
        if ((size_t)fa.maxDynamicSharedSizeBytes >= need) return DPD_OK;
        DPD_CU(cudaFuncSetAttribute(k_pair<P, T, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)need));
        return DPD_OK;
    }

    // Shared memory of the persistent step kernel (the plain pair kernel's) and
    // its co-resident grid: every block must be resident at once.
    template <int T>
    int set_persist_t() {
        persist_grid_ = 0;
        if (smem_n_ > 48 * 1024) {
            cudaFuncAttributes fa;
            DPD_CU(cudaFuncGetAttributes(&fa, k_steps<P, T>));
            if ((size_t)fa.maxDynamicSharedSizeBytes < smem_n_)
                DPD_CU(cudaFuncSetAttribute(k_steps<P, T>,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem_n_));
        }
        int dev = 0, nsm = 0, per_sm = 0;
        DPD_CU(cudaGetDevice(&dev));
        DPD_CU(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
        DPD_CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_steps<P, T>, T, smem_n_));
        persist_grid_ = per_sm * nsm;
        return DPD_OK;
    }

    template <int T>
    int launch_persistent_t(const StepArgs<P> &sa) {
        // as many blocks as the largest phase can use, at most the co-resident
        // grid: the pair phase takes one brick per block at a time, the bead
        // phases a few beads per thread
        const int want = std::max({sa.nbricks, (sa.nbeads + 4 * T - 1) / (4 * T), sa.ntiles, 1});
        const int grid = std::min(std::min(persist_grid_, want), BAR_GROUP * BAR_MAX_GROUPS);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid);
        cfg.blockDim = dim3((unsigned)T);
        cfg.dynamicSmemBytes = smem_n_;
        cfg.stream = stream_;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        cfg.attrs = at;
        cfg.numAttrs = 1;
        DPD_CU(cudaLaunchKernelEx(&cfg, k_steps<P, T>, sa));
        ++launches_;
        return DPD_OK;
    }

    // All steps of one dpd_step call in one cooperative launch (persist.cuh);
    // the kernel runs the same phases in the same order as enqueue_step.
    int launch_persistent(int64_t nsteps) {
        StepArgs<P> sa;
        std::memset(&sa, 0, sizeof(sa));
        sa.nsteps = (int)nsteps;
        sa.nbeads = used_beads_;
        sa.ncells = used_cells_;
        sa.nbricks = used_bricks_;
        sa.ntiles = (used_cells_ + SCAN_B - 1) / SCAN_B;
        sa.with_update = 1;
        UpdArgs<P> &ua = sa.upd;
        ua.b_lo = 0;
        ua.b_hi = used_beads_;
        ua.sys = sys_;
        ua.bsys = bsys_;
        ua.sys1 = sys1();
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
        for (int p = 0; p < 2; ++p) {
            const int old = cur_ ^ p, nxt = old ^ 1;
            ScatterArgs<P> &sc = sa.sc[p];
            sc.b_lo = 0;
            sc.b_hi = used_beads_;
            sc.sys = sys_;
            sc.bsys = bsys_;
            sc.sys1 = sys1();
            sc.key_tmp = key_tmp_;
            sc.rank = rank_;
            sc.cell_start = cell_start_;
            sc.id_old = id_[old];
            sc.srcid = srcid_;
            GatherArgs<P> &ga = sa.ga[p];
            ga.b_lo = 0;
            ga.b_hi = used_beads_;
            ga.sys = sys_;
            ga.bsys = bsys_;
            ga.srcid = srcid_;
            ga.cell_start = cell_start_;
            ga.pos_tmp = pos_tmp_;
            ga.vel_old = vel_[old];
            ga.frc_old = frc_[old];
            ga.key_tmp = key_tmp_;
            ga.pos = pos_;
            ga.vel = vel_[nxt];
            ga.frc = frc_[nxt];
            ga.vt = vt_;
            ga.key = key_;
            ga.id = id_[nxt];
            ga.inv_perm = used_bonds_ > 0 ? inv_perm_ : nullptr;
            ga.sys1 = sys1();
            ga.from = rank_;
            BondArgs<P> &ba = sa.bo[p];
            ba.b_lo = 0;
            ba.b_hi = used_beads_;
            ba.sys = sys_;
            ba.bsys = bsys_;
            ba.fpair = frc_[nxt];   // the pair phase writes the new force buffer
            ba.pos = pos_;
            ba.key = key_;
            ba.id = id_[nxt];
            ba.inv_perm = inv_perm_;
            ba.bptr = used_bonds_ > 0 ? bptr_ : nullptr;
            ba.bpartner = bpartner_;
            ba.bpar = bpar_;
            ba.sys1 = sys1();
            ba.from = rank_;
            ba.vel_old = vel_[old];
            ba.frc_old = frc_[old];
            ba.vel = vel_[nxt];
            ba.frc = frc_[nxt];
            ba.ev = ev_;
            ba.pos_tmp = pos_tmp_;
            ba.key_tmp = key_tmp_;
            ba.rank = rank_;
            ba.count = count_;
            ba.counter = counter_;
            ba.status = status_;
        }
        PairLaunch<P> &pl = sa.pl[0];
        pl.sys = sys_;
        pl.brick_sys = brick_sys_;
        pl.sys1 = sys1();
        pl.br_lo = 0;
        pl.capmax = capmax_;
        pl.Xmax = xmax_;
        pl.ntmax = ntmax_;
        pl.lntab = lntab_;
        pl.pos = pos_;
        pl.vt = vt_;
        pl.key = key_;
        pl.cell_start = cell_start_;
        pl.ev = ev_;
        pl.atab = atab_;
        pl.counter = counter_;
        pl.status = status_;
        sa.pl[1] = pl;
        for (int p = 0; p < 2; ++p) sa.pl[p].fpair = sa.bo[p].frc;   // into the step's force buffer
        sa.count = count_;
        sa.bsum = bsum_;
        sa.cell_start = cell_start_;
        sa.bar = bar_;
        sa.budget = kBarrierBudget;
        sa.status = status_;
        DPD_CU(cudaMemsetAsync(bar_, 0, sizeof(GridBar), stream_));
        int rc;
        switch (T_) {
            case 64: rc = launch_persistent_t<64>(sa); break;
            case 256: rc = launch_persistent_t<256>(sa); break;
            default: rc = launch_persistent_t<128>(sa); break;
        }
        if (rc) return rc;
        DPD_CU(cudaGetLastError());
        if (nsteps & 1) cur_ ^= 1;
        return DPD_OK;
    }

    template <int T, bool S>
    int launch_pair_t(const PairLaunch<P> &pl, int nbr) {
        DPD_CU(launch_pdl(k_pair<P, T, S>, nbr, T, S ? smem_ : smem_n_, stream_, pl));
        ++launches_;
        DPD_CU(cudaGetLastError());
        return DPD_OK;
    }

    // pair forces of bricks [br_lo, br_lo + nbr) into `out` (new order)
    int launch_pair(bool sample, int br_lo, int nbr, vec4 *out) {
        if (nbr <= 0) return DPD_OK;
        PairLaunch<P> pl;
        pl.sys = sys_;
        pl.brick_sys = brick_sys_;
        pl.sys1 = sys1();
        pl.br_lo = br_lo;
        pl.capmax = capmax_;
        pl.Xmax = xmax_;
        pl.ntmax = ntmax_;
        pl.lntab = lntab_;
        pl.pos = pos_;
        pl.vt = vt_;
        pl.key = key_;
        pl.cell_start = cell_start_;
        pl.fpair = out;
        pl.ev = ev_;
        pl.atab = atab_;
        pl.counter = counter_;
        pl.status = status_;
        switch (T_) {
            case 64:
                return sample ? launch_pair_t<64, true>(pl, nbr) : launch_pair_t<64, false>(pl, nbr);
            case 256:
                return sample ? launch_pair_t<256, true>(pl, nbr) : launch_pair_t<256, false>(pl, nbr);
            default:
                return sample ? launch_pair_t<128, true>(pl, nbr) : launch_pair_t<128, false>(pl, nbr);
        }
    }

    // cell division of beads [b_lo, b_hi) / cells [c_lo, c_hi), from the
    // `old` velocity/force/id buffers into the `nxt` ones
    int enqueue_sort(int b_lo, int b_hi, int c_lo, int c_hi, int old, int nxt,
                     bool move_vf = false) {
        const int C = c_hi - c_lo, nb = (C + SCAN_B - 1) / SCAN_B;
        DPD_CU(launch_pdl(k_scan1, nb, SCAN_T, 0, stream_, count_ + c_lo, C, bsum_));
        DPD_CU(launch_pdl(k_scan3b, nb, SCAN_T, 0, stream_, count_ + c_lo, C,
                          (const uint32_t *)bsum_, cell_start_ + c_lo, (uint32_t)b_lo));
        ScatterArgs<P> sa;
        sa.b_lo = b_lo;
        sa.b_hi = b_hi;
        sa.sys = sys_;
        sa.bsys = bsys_;
        sa.sys1 = sys1();
        sa.key_tmp = key_tmp_;
        sa.rank = rank_;
        sa.cell_start = cell_start_;
        sa.id_old = id_[old];
        sa.srcid = srcid_;
        DPD_CU(launch_pdl(k_scatter<P>, blocks(b_hi - b_lo), 256, 0, stream_, sa));
        GatherArgs<P> ga;
        ga.b_lo = b_lo;
        ga.b_hi = b_hi;
        ga.sys = sys_;
        ga.bsys = bsys_;
        ga.srcid = srcid_;
        ga.cell_start = cell_start_;
        ga.pos_tmp = pos_tmp_;
        ga.vel_old = vel_[old];
        ga.frc_old = frc_[old];
        ga.key_tmp = key_tmp_;
        ga.pos = pos_;
        ga.vel = vel_[nxt];
        ga.frc = frc_[nxt];
        ga.vt = vt_;
        ga.key = key_;
        ga.id = id_[nxt];
        ga.inv_perm = used_bonds_ > 0 ? inv_perm_ : nullptr;
        ga.sys1 = sys1();
        ga.from = rank_;   // the arrival ranks are consumed by the scatter
        if (move_vf) DPD_CU(launch_pdl(k_gather<P, true>, blocks(b_hi - b_lo), 256, 0, stream_, ga));
        else DPD_CU(launch_pdl(k_gather<P, false>, blocks(b_hi - b_lo), 256, 0, stream_, ga));
        launches_ += 4;
        DPD_CU(cudaGetLastError());
        return DPD_OK;
    }

    // bonds (+ velocity update unless init) over beads [b_lo, b_hi)
    int enqueue_bonds(bool init, bool sample, int b_lo, int b_hi, bool fuse = false,
                      bool obs_only = false) {
        BondArgs<P> ba;
        ba.b_lo = b_lo;
        ba.b_hi = b_hi;
        ba.sys = sys_;
        ba.bsys = bsys_;
        ba.fpair = frc_[cur_];   // the pair kernel wrote the new force buffer
        ba.pos = pos_;
        ba.key = key_;
        ba.id = id_[cur_];
        ba.inv_perm = inv_perm_;
        ba.bptr = used_bonds_ > 0 ? bptr_ : nullptr;
        ba.bpartner = bpartner_;
        ba.bpar = bpar_;
        ba.sys1 = sys1();
        ba.from = rank_;                  // source slots recorded by the sort's gather
        ba.vel_old = vel_[cur_ ^ 1];
        ba.frc_old = frc_[cur_ ^ 1];
        ba.vel = vel_[cur_];
        ba.frc = frc_[cur_];
        ba.ev = ev_;
        ba.pos_tmp = pos_tmp_;
        ba.key_tmp = key_tmp_;
        ba.rank = rank_;
        ba.count = count_;
        ba.counter = counter_;
        ba.status = status_;
        const int g = blocks(b_hi - b_lo);
        if (obs_only) {
            DPD_CU(launch_pdl(k_bond_obs<P>, g, 256, 0, stream_, ba));
        } else if (init) {
            if (sample) DPD_CU(launch_pdl(k_bond_vel<P, true, true>, g, 256, 0, stream_, ba));
            else DPD_CU(launch_pdl(k_bond_vel<P, true, false>, g, 256, 0, stream_, ba));
        } else if (fuse) {
            DPD_CU(launch_pdl(k_bond_vel<P, false, false, true>, g, 256, 0, stream_, ba));
        } else {
            if (sample) DPD_CU(launch_pdl(k_bond_vel<P, false, true>, g, 256, 0, stream_, ba));
            else DPD_CU(launch_pdl(k_bond_vel<P, false, false>, g, 256, 0, stream_, ba));
        }
        ++launches_;
        DPD_CU(cudaGetLastError());
        return DPD_OK;
    }

    // FP64 observables of systems rsys[k0 .. k0+nk) from chunks [r0, r0+nr)
    int enqueue_reduce(int r0, int nr, int k0, int nk, bool accumulate) {
        if (nr <= 0 || nk <= 0) return DPD_OK;
        DPD_CU(launch_pdl(k_reduce<P>, nr, RED_T, 0, stream_, (const int2 *)(rmap_ + r0),
                          (const vec4 *)vel_[cur_], (const vec4 *)ev_, partial_ + r0 * RED_K));
        DPD_CU(launch_pdl(k_reduce_final<P>, nk, RED_T, 0, stream_, (const int4 *)(rsys_ + k0),
                          (const SysDesc<P> *)sys_, (const double *)partial_, obs_, acc_,
                          accumulate ? 1 : 0, status_));
        launches_ += 2;
        DPD_CU(cudaGetLastError());
        return DPD_OK;
    }

    // One step of every resident system.  with_update: run the position update
    // here (else the previous step's bond kernel did it); fuse: this step's bond
    // kernel does the next step's update (never on a sampled step).
    int enqueue_step(bool sample, bool accumulate, bool capturing, bool with_update, bool fuse) {
        int rc = mark(0, capturing);
        if (rc) return rc;
        UpdArgs<P> ua;
        ua.b_lo = 0;
        ua.b_hi = used_beads_;
        ua.sys = sys_;
        ua.bsys = bsys_;
        ua.sys1 = sys1();
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
        if (with_update) {
            DPD_CU(launch_pdl(k_update<P>, blocks(used_beads_), 256, 0, stream_, ua));
            ++launches_;
            DPD_CU(cudaGetLastError());
        }
        const int nxt = cur_ ^ 1;
        if ((rc = enqueue_sort(0, used_beads_, 0, used_cells_, cur_, nxt))) return rc;
        cur_ = nxt;
        if ((rc = mark(1, capturing)) || (rc = launch_pair(sample, 0, used_bricks_, frc_[cur_])) ||
            (rc = mark(2, capturing)) ||
            (rc = enqueue_bonds(false, sample, 0, used_beads_, fuse && !sample)))
            return rc;
        if (sample && (rc = enqueue_reduce(0, nred_all_, 0, nrsys_all_, accumulate))) return rc;
        return mark(3, capturing);
    }

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

    void drop_graphs() {
        for (auto &row : graphs_)
            for (auto &g : row) {
                if (g.exec) cudaGraphExecDestroy(g.exec);
                if (g.graph) cudaGraphDestroy(g.graph);
                g = GraphSlot();
            }
    }

    // One captured step per (parity, variant): the ping-pong buffers swap
    // every step, so a graph is valid for the parity it was captured at; any
    // change of the pools' membership drops the graphs.
    int launch_graph(int variant) {
        GraphSlot &g = graphs_[cur_][variant];
        if (!g.exec) {
            const int cur0 = cur_;
            const int64_t l0 = launches_;
            cudaGraph_t graph = nullptr;
            DPD_CU(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal));
            const int base = variant % 3;
            int rc = enqueue_step(base == 2, base == 2, true, variant < 3, base == 0);
            cudaError_t e = cudaStreamEndCapture(stream_, &graph);
            cur_ = cur0;   // capture did not execute anything
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

    BatchConfig bc_;
    int NB_ = 0, NC_ = 0, NBR_ = 0, NBD_ = 0, NS_ = 0, NRB_ = 0, T_ = 128;
    cudaStream_t stream_ = nullptr;
    bool own_stream_ = false;
    static constexpr int IO_MAXCH = 8, IO_CHUNK = 1 << 18;
    cudaStream_t xfer_ = nullptr;          // host <-> device state copies
    cudaEvent_t xev_[IO_MAXCH + 1] = {};
    std::vector<void *> allocs_;
    std::vector<SysHost> hs_;
    std::vector<SysDesc<P>> hsys_;
    std::vector<int> order_;               // live systems in pool order
    int used_beads_ = 0, used_cells_ = 0, used_bricks_ = 0, used_bonds_ = 0;
    int nred_all_ = 0, nrsys_all_ = 0;
    int capmax_ = 0, xmax_ = 0, ntmax_ = 1;
    size_t smem_ = 0, smem_n_ = 0;   // pair-kernel shared memory: sampled, plain
    vec4 *pos_ = nullptr, *pos_tmp_ = nullptr, *vel_[2] = {nullptr, nullptr},
         *frc_[2] = {nullptr, nullptr}, *vt_ = nullptr, *ev_ = nullptr;
    uint32_t *key_ = nullptr, *key_tmp_ = nullptr, *rank_ = nullptr;
    uint2 *srcid_ = nullptr;
    int32_t *id_[2] = {nullptr, nullptr}, *inv_perm_ = nullptr, *types_ = nullptr;
    LnTab *lntab_ = nullptr;
    int *bsys_ = nullptr, *brick_sys_ = nullptr, *old_bead0_ = nullptr;
    uint32_t *count_ = nullptr, *cell_start_ = nullptr, *bsum_ = nullptr;
    SysDesc<P> *sys_ = nullptr;
    long long *counter_ = nullptr;
    int *status_ = nullptr;
    real *atab_ = nullptr;
    int32_t *bptr_ = nullptr, *bpartner_ = nullptr;
    vec4 *bpar_ = nullptr;
    struct UploadBufs {   // host data of an upload whose copies are in flight
        UploadBufs(std::vector<real> &&a_, std::vector<int32_t> &&b_, std::vector<vec4> &&p_)
            : a(std::move(a_)), bp(std::move(b_)), par(std::move(p_)) {}
        std::vector<real> a;
        std::vector<int32_t> bp;
        std::vector<vec4> par;
    };
    std::vector<std::shared_ptr<UploadBufs>> upload_keep_;
    bool repack_pending_ = false;
    GridBar *bar_ = nullptr;               // the persistent kernel's grid barrier
    int persist_grid_ = 0;                 // its co-resident grid (0: not available)
    // clock cycles a block of the persistent kernel waits at one grid barrier
    // before it gives up (about two seconds at 2 GHz)
    static constexpr long long kBarrierBudget = 4000000000LL;
    int2 *rmap_ = nullptr;
    int4 *rsys_ = nullptr;
    double *partial_ = nullptr, *obs_ = nullptr, *acc_ = nullptr, *io_ = nullptr;
    size_t io_n_ = 0;
    int cur_ = 0;
    int64_t launches_ = 0;
    int status_host_ = 0;
    GraphSlot graphs_[2][6];   // [parity][variant]: fused/last/accumulating x with/without update
    cudaEvent_t ph_[4] = {nullptr, nullptr, nullptr, nullptr};
    std::vector<cudaEvent_t> prof_ev_;
    int64_t prof_max_ = 0, prof_n_ = 0;
    bool prof_on_ = false;
};

}  // namespace dpd
