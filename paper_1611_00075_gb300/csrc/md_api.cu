// md_api.cu -- the C ABI (include/md_gb300.h): argument checks, device
// memory, and the order in which kernels are enqueued for each call.
//
// Time stepping (Sec. 3.3, velocity-Verlet): the first half kick and drift of
// a run use the forces of the previous evaluation; each later force kernel
// applies the closing half kick of its step merged with the opening half kick
// of the next one, then drifts; the last step only applies its closing half
// kick.  Before every force evaluation a rebuild chain (binning + list) is
// enqueued that runs only when the device rebuild flag is set, so the host
// never waits for the half-skin test.  md_step reads the device status once
// at the end; a list overflow found there is repaired and the remaining steps
// are re-enqueued from the step that stopped.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "md_internal.cuh"

using namespace mdg;

namespace {

thread_local std::string g_thread_error;

md_status fail(md_system *h, md_status st, const std::string &msg) {
    if (h) h->last_error = msg;
    else g_thread_error = msg;
    return st;
}

#define MD_CK(call)                                                                        \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(h, MD_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

template <class T>
cudaError_t dalloc(T **p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void **)p, count * sizeof(T));
}

bool is_int_valued(double x, int lo, int hi) {
    return std::isfinite(x) && std::floor(x) == x && x >= lo && x <= hi;
}

md_status check_params(const md_params *p, int64_t n, const double *box, std::string *why) {
    auto bad = [&](const char *m) { *why = m; return MD_ERR_INVALID; };
    if (n < 1) return bad("n must be >= 1");
    if (n >= kMaxAtoms) return bad("n must be below 2^27");
    if (p->potential != MD_POT_LJ && p->potential != MD_POT_SC && p->potential != MD_POT_EAM)
        return bad("unknown potential");
    if (p->precision != MD_FP64 && p->precision != MD_MIXED) return bad("unknown precision");
    if (p->force_variant < MD_FORCE_FULL || p->force_variant > MD_FORCE_PAIRED)
        return bad("unknown force_variant");
    if (p->scheduler < MD_SCHED_GRID || p->scheduler > MD_SCHED_DYNAMIC)
        return bad("unknown scheduler");
    if (p->rebuild_every < 0) return bad("rebuild_every must be >= 0");
    if (p->max_neighbors < 0) return bad("max_neighbors must be >= 0");
    if (!(p->rc > 0) || !(p->skin >= 0) || !(p->dt > 0) || !(p->mass > 0) ||
        !std::isfinite(p->rc + p->skin + p->dt + p->mass))
        return bad("rc, dt, mass must be > 0 and skin >= 0");
    if (p->potential != MD_POT_EAM &&
        (!(p->eps > 0) || !(p->sigma > 0) || !std::isfinite(p->eps + p->sigma)))
        return bad("eps and sigma must be > 0");
    if (p->potential == MD_POT_SC) {
        if (!(p->c > 0) || !std::isfinite(p->c)) return bad("Sutton-Chen c must be > 0");
        if (!is_int_valued(p->n_exp, 1, 30) || !is_int_valued(p->m_exp, 1, 30))
            return bad("Sutton-Chen n and m must be integers in [1, 30]");
    }
    const double rl = p->rc + p->skin;
    double ncells = 1.0;
    for (int d = 0; d < 3; ++d) {
        if (!(box[d] > 0) || !std::isfinite(box[d])) return bad("box sides must be > 0");
        double q = std::floor(box[d] / rl);
        if (q < 3) return bad("each box side must hold at least 3 list radii (rc + skin)");
        ncells *= q;
    }
    if (ncells > 2.0e9) return bad("too many cells");
    return MD_OK;
}

void free_all(md_system *h) {
    auto F = [](void *p) { if (p) cudaFree(p); };
    for (int b = 0; b < 2; ++b) { F(h->xr64[b]); F(h->xq[b]); }
    F(h->xq_build); F(h->xabs); F(h->v); F(h->f); F(h->e_atom); F(h->orig); F(h->cell);
    F(h->cell_start); F(h->cell_count); F(h->new_cell); F(h->slot); F(h->src); F(h->key);
    F(h->scan_bsum); F(h->tmp_abs); F(h->tmp_v); F(h->nlist); F(h->ncount);
    F(h->rho); F(h->dF32); F(h->dF64); F(h->xqf); F(h->partials); F(h->red_out); F(h->ds);
    F(h->exp_tmp); F(h->type_orig);
    F(h->cl_icnt); F(h->cl_jcnt); F(h->cl_ioff); F(h->cl_joff); F(h->cl_bsum); F(h->cl_icl);
    F(h->cl_icell); F(h->cl_jbox); F(h->cl_ntot); F(h->cl_list); F(h->cl_row);
    F(h->ps_cnt); F(h->ps_start); F(h->ps_bsum); F(h->ps_atom); F(h->ps_list); F(h->ps_count);
    F(h->ov_cell_outer); F(h->ov_flag); F(h->ov_pos); F(h->ov_bsum); F(h->ov_gidx);
    F(h->ov_bidx); F(h->ov_nb); F(h->ov_send); F(h->ov_recv);
    if (h->ov_stream) cudaStreamDestroy(h->ov_stream);
    for (cudaEvent_t ev : h->ov_ev)
        if (ev) cudaEventDestroy(ev);
    F(h->part_bounds); F(h->cell_cost); F(h->part_scratch); F(h->cell_X); F(h->cell_pred);
    F(h->cell_cycles); F(h->cta_cycles); F(h->samp_flag); F(h->samp_bsum); F(h->samp_X);
    F(h->samp_y); F(h->mlp_P); F(h->mlp_G); F(h->mlp_m); F(h->mlp_v); F(h->mlp_scratch);
    F(h->mlp_loss);
    F(h->grids); F(h->ctab); F(h->atom_off); F(h->rep); F(h->shifts32); F(h->rep_pe);
    F(h->rep_ke);
    if (h->ds_host) cudaFreeHost(h->ds_host);
    if (h->red_host) cudaFreeHost(h->red_host);
}

void drop_graphs(md_system *h);

// Cluster tables and a cluster list of cl_cap entries per i-cluster, sized
// from the largest cell occupancy seen (a quarter of headroom).
cudaError_t alloc_cluster(md_system *h, int max_cell) {
    const size_t C = (size_t)h->g.ncells;
    const int64_t rows = cluster_rows(h->n, h->g.ncells);
    const int64_t jrows = h->n / 4 + h->g.ncells + 1;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    if (!h->cl_icnt) {
        A(dalloc(&h->cl_icnt, C)); A(dalloc(&h->cl_jcnt, C)); A(dalloc(&h->cl_ioff, C + 1));
        A(dalloc(&h->cl_joff, C + 1)); A(dalloc(&h->cl_bsum, C / (kBlock * 8) + 4));
        A(dalloc(&h->cl_icl, (size_t)rows)); A(dalloc(&h->cl_icell, (size_t)rows));
        A(dalloc(&h->cl_jbox, 2 * (size_t)jrows)); A(dalloc(&h->cl_ntot, 2));
        A(dalloc(&h->cl_row, (size_t)rows));
    }
    const int cap = cluster_cap(max_cell + max_cell / 4 + 4);
    if (e == cudaSuccess && (cap > h->cl_cap || !h->cl_list)) {
        if (h->cl_list) cudaFree(h->cl_list);
        h->cl_list = nullptr;
        h->cl_cap = cap;
        A(dalloc(&h->cl_list, (size_t)rows * cap));
    }
    return e;
}

// Slot tables, then a union list of ps_cap entries per slot; cap == 0 keeps
// the list (tables only).
cudaError_t alloc_pair(md_system *h, int cap) {
    const size_t C = (size_t)h->g.ncells;
    const int64_t smax = pair_slots_max(h->n, h->g.ncells);
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    if (!h->ps_cnt) {
        A(dalloc(&h->ps_cnt, C)); A(dalloc(&h->ps_start, C + 1));
        A(dalloc(&h->ps_bsum, C / (kBlock * 8) + 4)); A(dalloc(&h->ps_atom, (size_t)smax));
        A(dalloc(&h->ps_count, (size_t)smax));
    }
    if (e == cudaSuccess && cap > 0 && (cap != h->ps_cap || !h->ps_list)) {
        drop_graphs(h);  // captured steps hold the old list pointer and capacity
        if (h->ps_list) cudaFree(h->ps_list);
        h->ps_list = nullptr;
        h->ps_cap = cap;
        A(dalloc(&h->ps_list, (size_t)((smax + 31) / 32) * 32 * (size_t)cap));
    }
    return e;
}

int cap_for(int max_count);
md_status read_status(md_system *h);
md_status clear_status(md_system *h);

// Slot tables and union lists for the current binning, sized from a count
// pass when the list is new, regrown when a row overflows.
md_status pair_rebuild_now(md_system *h) {
    MD_CK(alloc_pair(h, 0));
    if (!h->ps_list) {
        MD_CK(launch_pair_build(h, false, false));
        md_status st = read_status(h);
        if (st != MD_OK) return st;
        if (h->ds_host->status != 0)
            return fail(h, (md_status)h->ds_host->status, "device error during slot list count");
        MD_CK(alloc_pair(h, std::max(cap_for(h->ds_host->pair_max), 8)));
    }
    for (int attempt = 0; attempt < 3; ++attempt) {
        MD_CK(launch_pair_build(h, true, false));
        md_status st = read_status(h);
        if (st != MD_OK) return st;
        if (h->ds_host->status == 0) return MD_OK;
        if (h->ds_host->status != MD_ERR_LIST_OVERFLOW)
            return fail(h, (md_status)h->ds_host->status, "device error during slot list build");
        st = clear_status(h);
        if (st != MD_OK) return st;
        MD_CK(alloc_pair(h, cap_for(h->ds_host->pair_max)));
    }
    return fail(h, MD_ERR_LIST_OVERFLOW, "slot list overflow could not be repaired");
}

cudaError_t alloc_list(md_system *h, int cap) {
    drop_graphs(h);  // captured steps hold the old list pointer and capacity
    if (h->nlist) cudaFree(h->nlist);
    h->nlist = nullptr;
    h->cap = cap;
    h->nlist_entries = (size_t)((h->n + 31) / 32) * 32 * (size_t)cap;
    cudaError_t e = dalloc(&h->nlist, h->nlist_entries);
    if (e == cudaSuccess && h->p.force_variant == MD_FORCE_CLUSTER)
        e = alloc_cluster(h, h->ds_host ? h->ds_host->max_cell : 32);
    return e;
}

int cap_for(int max_count) {
    int c = max_count + max_count / 4 + 8;
    return (c + 7) & ~7;
}

md_status read_status(md_system *h) {
    MD_CK(cudaMemcpyAsync(h->ds_host, h->ds, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                          h->stream));
    MD_CK(cudaStreamSynchronize(h->stream));
    return MD_OK;
}

md_status clear_status(md_system *h) {
    MD_CK(cudaMemsetAsync(&h->ds->status, 0, sizeof(int), h->stream));
    // a launch that stopped early may have left the tile queue mid-count
    MD_CK(cudaMemsetAsync(&h->ds->tile_counter, 0, 2 * sizeof(int), h->stream));
    return MD_OK;
}

// ---- per-launch timing: an event after each interval, summed at sync -------
enum { K_REBUILD = 0, K_FORCE = 1, K_INTEGRATE = 2, K_OTHER = 3 };

cudaError_t mark(md_system *h, int kind) {
    if (!h->timing) return cudaSuccess;
    if (h->ev_used == h->ev_pool.size()) {
        cudaEvent_t e;
        cudaError_t r = cudaEventCreate(&e);
        if (r != cudaSuccess) return r;
        h->ev_pool.push_back(e);
        h->ev_kind.push_back(K_OTHER);
    }
    h->ev_kind[h->ev_used] = kind;
    return cudaEventRecord(h->ev_pool[h->ev_used++], h->stream);
}

// after a synchronize: accumulate intervals ev[k-1] -> ev[k] by the kind of
// ev[k], for the first `upto` events (all of them by default); the rest are
// dropped
void harvest(md_system *h, size_t upto = SIZE_MAX) {
    const size_t used = std::min(upto, h->ev_used);
    for (size_t k = 1; k < used; ++k) {
        float ms = 0.f;
        if (h->ev_kind[k] >= 0 && cudaEventElapsedTime(&ms, h->ev_pool[k - 1], h->ev_pool[k]) == cudaSuccess) {
            h->ms_kind[h->ev_kind[k]] += ms;
            h->n_kind[h->ev_kind[k]] += 1;
        }
    }
    h->ev_used = 0;
}

// ---- persistent scheduler ----------------------------------------------------

// The persistent kernel serves the mixed-precision Lennard-Jones full-list
// force pass; every other combination uses the one-thread-per-atom grid.
bool persistent_path(const md_system *h) {
    return h->p.scheduler != MD_SCHED_GRID && h->p.potential == MD_POT_LJ &&
           (h->p.force_variant == MD_FORCE_FULL || h->p.force_variant == MD_FORCE_PAIRED);
}

bool uses_partition(const md_system *h) {
    return persistent_path(h) &&
           (h->p.scheduler == MD_SCHED_PAIRCOUNT || h->p.scheduler == MD_SCHED_MLP);
}

// Resident CTAs and ranges per CTA of the persistent kernel of the current
// force layout (the two-atom kernel runs fewer, larger CTAs per SM).
void sched_shape(md_system *h) {
    if (!h->sched_tail_set)
        h->sched_tail_pct = h->p.force_variant == MD_FORCE_PAIRED ? kTailPctPaired : kTailPctDefault;
    if (h->sched_sms <= 0) return;
    const bool paired = (h->p.force_variant == MD_FORCE_PAIRED);
    h->sched_ctas = h->sched_sms * persist_ctas_per_sm(h->p.precision == MD_FP64, paired);
    // ranges of about kTilesPerRange tiles of the layout's work items (atoms,
    // or slots of two atoms)
    const int64_t items = paired ? (h->n + 1) / 2 : h->n;
    h->sched_rounds = h->sched_rounds_set > 0 ? h->sched_rounds_set : sched_rounds(items, h->sched_ctas);
}

// Buffers of the scheduler and the cost model, allocated on first use.
md_status ensure_sched(md_system *h) {
    if (h->part_bounds) return MD_OK;
    drop_graphs(h);
    int dev = 0, sms = 0;
    MD_CK(cudaGetDevice(&dev));
    MD_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    h->sched_sms = sms;
    // buffers sized for the largest CTA count of any persistent kernel
    const int ctas_max = sms * std::max(persist_ctas_per_sm(h->p.precision == MD_FP64, false),
                                        persist_ctas_per_sm(false, true));
    h->sched_ctas = ctas_max;
    const size_t C = (size_t)h->g.ncells;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    h->sched_rounds = h->sched_rounds_set > 0 ? h->sched_rounds_set : sched_rounds(h->n, h->sched_ctas);
    // room for the largest partition md_set_schedule allows
    A(dalloc(&h->part_bounds, (size_t)sched_parts(h->sched_ctas, kSchedRounds, kTailPctMax) + 1));
    A(dalloc(&h->cell_cost, C));
    A(dalloc(&h->part_scratch, C + 1 + C / (kBlock * 8) + 8));
    A(dalloc(&h->cell_X, 3 * C));
    A(dalloc(&h->cell_pred, C));
    A(dalloc(&h->cell_cycles, C));
    A(dalloc(&h->cta_cycles, (size_t)ctas_max));
    A(dalloc(&h->samp_flag, 2 * (C + 1) + 2));  // flags, their scan, sample count
    A(dalloc(&h->samp_bsum, C / (kBlock * 8) + 8));
    A(dalloc(&h->samp_X, 3 * C));
    A(dalloc(&h->samp_y, C));
    A(dalloc(&h->mlp_P, kMlpParams));
    A(dalloc(&h->mlp_G, kMlpParams));
    A(dalloc(&h->mlp_m, kMlpParams));
    A(dalloc(&h->mlp_v, kMlpParams));
    A(dalloc(&h->mlp_scratch, mlp_grad_scratch_floats((long long)C)));
    A(dalloc(&h->mlp_loss, 1));
    if (e != cudaSuccess)
        return fail(h, e == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA,
                    std::string("scheduler allocation: ") + cudaGetErrorString(e));
    sched_shape(h);
    MD_CK(launch_mlp_init(h->mlp_P, 0x1611000075ull, h->stream));
    MD_CK(cudaMemsetAsync(h->mlp_m, 0, kMlpParams * sizeof(float), h->stream));
    MD_CK(cudaMemsetAsync(h->mlp_v, 0, kMlpParams * sizeof(float), h->stream));
    h->mlp_t = 0;
    return MD_OK;
}

// Cost estimate and equal-cost partition of the cells over the persistent
// CTAs; part of the rebuild chain (gated) or run right away.
md_status enqueue_sched_prep(md_system *h, bool gated) {
    if (!uses_partition(h)) return MD_OK;
    // the cost model learns the mixed kernel's timings; the float64 path
    // partitions by pair count under either static scheduler
    const bool pc = (h->p.scheduler == MD_SCHED_PAIRCOUNT) || h->p.precision == MD_FP64;
    MD_CK(launch_cell_features(h, pc, gated));
    if (!pc) MD_CK(launch_predict_costs(h, gated));
    MD_CK(launch_partition_cells(h, gated));
    h->launches += pc ? 5 : 7;
    return MD_OK;
}

// Rebuild chain enqueued before a force evaluation.  gated: runs only if the
// device flag asks for it.
md_status enqueue_rebuild(md_system *h, bool gated) {
    MD_CK(launch_bin(h, gated));
    if (h->p.force_variant == MD_FORCE_PAIRED) {
        MD_CK(launch_pair_build(h, true, gated));
        h->launches += kBinLaunches + 8;  // binning, slot tables and lists, finish
    } else {
        MD_CK(launch_build_list(h, true, gated));
        h->launches += kBinLaunches + 3;  // binning, list reset and build, finish
    }
    if (h->ov_on) {
        MD_CK(launch_overlap_index(h, gated));
        h->launches += 5;
    }
    if (h->p.force_variant == MD_FORCE_CLUSTER) {
        MD_CK(launch_cluster_build(h, gated));
        h->launches += 9;
    }
    md_status st = enqueue_sched_prep(h, gated);
    if (st != MD_OK) return st;
    MD_CK(launch_finish_rebuild(h, gated));
    MD_CK(mark(h, K_REBUILD));
    return MD_OK;
}

// Host-driven rebuild with capacity repair (explicit calls and create).
md_status rebuild_now(md_system *h, bool size_from_count) {
    MD_CK(launch_bin(h, false));
    if (h->p.force_variant == MD_FORCE_PAIRED) {
        // the slot lists carry the force pass; per-atom rows are built on
        // demand for export (atom_list_for_export)
        md_status st = pair_rebuild_now(h);
        if (st != MD_OK) return st;
        st = enqueue_sched_prep(h, false);
        if (st != MD_OK) return st;
        MD_CK(launch_finish_rebuild(h, false));
        h->list_valid = true;
        h->forces_valid = false;
        return MD_OK;
    }
    if (size_from_count || h->nlist == nullptr) {
        MD_CK(launch_build_list(h, false, false));
        md_status st = read_status(h);
        if (st != MD_OK) return st;
        if (h->ds_host->status != 0)
            return fail(h, (md_status)h->ds_host->status, "device error during list count");
        int cap = h->p.max_neighbors > 0 ? ((h->p.max_neighbors + 3) & ~3) : cap_for(h->ds_host->max_count);
        cap = std::max(cap, 8);
        if (cap != h->cap || h->nlist == nullptr) MD_CK(alloc_list(h, cap));
    }
    for (int attempt = 0; attempt < 3; ++attempt) {
        MD_CK(launch_build_list(h, true, false));
        md_status st = read_status(h);
        if (st != MD_OK) return st;
        if (h->ds_host->status == 0) break;
        if (h->ds_host->status != MD_ERR_LIST_OVERFLOW)
            return fail(h, (md_status)h->ds_host->status, "device error during list build");
        if (h->p.max_neighbors > 0)
            return fail(h, MD_ERR_LIST_OVERFLOW, "neighbour count exceeds max_neighbors");
        st = clear_status(h);
        if (st != MD_OK) return st;
        MD_CK(alloc_list(h, cap_for(h->ds_host->max_count)));
    }
    if (h->ov_on) MD_CK(launch_overlap_index(h, false));
    if (h->p.force_variant == MD_FORCE_CLUSTER) {
        md_status st = read_status(h);  // the binning's largest cell sizes the cluster list
        if (st != MD_OK) return st;
        MD_CK(alloc_cluster(h, h->ds_host->max_cell));
        MD_CK(launch_cluster_build(h, false));
        st = read_status(h);
        if (st != MD_OK) return st;
        if (h->ds_host->status != 0)
            return fail(h, (md_status)h->ds_host->status, "device error during cluster build");
    }
    md_status st = enqueue_sched_prep(h, false);
    if (st != MD_OK) return st;
    MD_CK(launch_finish_rebuild(h, false));
    h->list_valid = true;
    h->forces_valid = false;
    return MD_OK;
}

// Per-atom rows for export under MD_FORCE_PAIRED, whose rebuilds build the
// slot lists only: the list of the positions of the last build (xq_build,
// xabs), rebuilt when a build happened since the rows were last made.
md_status atom_list_for_export(md_system *h) {
    md_status st = read_status(h);
    if (st != MD_OK) return st;
    if (h->nlist != nullptr && h->atom_list_at == h->ds_host->builds) return MD_OK;
    MD_CK(launch_build_list(h, false, false, h->xq_build));
    st = read_status(h);
    if (st != MD_OK) return st;
    if (h->ds_host->status != 0)
        return fail(h, (md_status)h->ds_host->status, "device error during list count");
    int cap = h->p.max_neighbors > 0 ? ((h->p.max_neighbors + 3) & ~3) : cap_for(h->ds_host->max_count);
    cap = std::max(cap, 8);
    if (cap != h->cap || h->nlist == nullptr) MD_CK(alloc_list(h, cap));
    MD_CK(launch_build_list(h, true, false, h->xq_build));
    st = read_status(h);
    if (st != MD_OK) return st;
    if (h->ds_host->status != 0)
        return fail(h, (md_status)h->ds_host->status, "device error during the export list build");
    h->atom_list_at = h->ds_host->builds;
    return MD_OK;
}

md_status enqueue_forces(md_system *h, int mode, bool energy, bool store_f) {
    if (h->p.potential == MD_POT_SC) {
        MD_CK(launch_sc_density(h));
        MD_CK(launch_sc_force(h, mode, energy, store_f));
        h->launches += 2;
    } else if (h->p.potential == MD_POT_EAM) {
        MD_CK(launch_eam_density(h));
        MD_CK(launch_eam_force(h, mode, energy, store_f));
        h->launches += 2;
    } else if (h->ov_on) {
        MD_CK(launch_overlap_forces(h, mode, energy, store_f));
        h->launches += 4;
    } else if (h->p.force_variant == MD_FORCE_CLUSTER) {
        MD_CK(launch_cluster_forces(h, mode, energy, store_f));
        h->launches += 1;
    } else if (h->p.force_variant == MD_FORCE_PAIRED) {
        if (persistent_path(h) && !energy)
            MD_CK(launch_lj_persist(h, mode, store_f, h->p.scheduler == MD_SCHED_DYNAMIC, false));
        else
            MD_CK(launch_pair_forces(h, mode, energy, store_f));
        h->launches += 1;
    } else if (h->p.force_variant != MD_FORCE_FULL) {
        int nl = 0;
        MD_CK(launch_lj_half(h, mode, energy, &nl));
        h->launches += nl;
    } else if (persistent_path(h) && !energy) {
        MD_CK(launch_lj_persist(h, mode, store_f, h->p.scheduler == MD_SCHED_DYNAMIC, false));
        h->launches += 1;
    } else {
        MD_CK(launch_lj(h, mode, energy, store_f));
        h->launches += 1;
    }
    MD_CK(mark(h, K_FORCE));
    return MD_OK;
}

// Forces at the current positions (rebuilding first if the flag is set).
md_status forces_now(md_system *h, bool energy) {
    if (h->timing) {
        h->ev_used = 0;
        MD_CK(mark(h, -1));
    }
    md_status st = enqueue_rebuild(h, true);
    if (st != MD_OK) return st;
    const size_t ev_rebuilt = h->ev_used;  // through the rebuild's mark
    st = enqueue_forces(h, FM_STORE, energy, true);
    if (st != MD_OK) return st;
    st = read_status(h);
    if (st != MD_OK) return st;
    if (h->ds_host->status == MD_ERR_LIST_OVERFLOW) {
        // the gated rebuild overflowed, so the force launch did nothing:
        // repair on the host (timed as one more rebuild) and evaluate again
        if (h->timing) h->ev_used = ev_rebuilt;
        st = clear_status(h);
        if (st != MD_OK) return st;
        st = rebuild_now(h, true);
        if (st != MD_OK) return st;
        MD_CK(mark(h, K_REBUILD));
        st = enqueue_forces(h, FM_STORE, energy, true);
        if (st != MD_OK) return st;
        st = read_status(h);
        if (st != MD_OK) return st;
    }
    if (h->timing) harvest(h);
    if (h->ds_host->status != 0)
        return fail(h, (md_status)h->ds_host->status, "device error during force evaluation");
    h->forces_valid = true;
    h->list_valid = true;
    return MD_OK;
}

__global__ void begin_steps_kernel(DevStatus *ds, int base) { ds->steps_done = base; }

// ---- CUDA graphs of one full step ---------------------------------------------
//
// The launches of a step that is neither the first nor the last of an md_step
// call -- the rebuild chain and the fused force + kick + drift -- are the
// same every step except for the double-buffer parity, so they are captured
// once per parity and replayed.  The rebuild chain sits in the body of a
// conditional (IF) node whose condition a one-thread kernel sets from the
// device's rebuild flag, so a step without a rebuild launches two kernels
// instead of the whole gated chain.  Kernels that decide on the device
// (status word, step counter) keep working under replay.  Any change of
// buffers or launch choice drops the graphs; capture needs a non-default
// stream.  With per-launch timing on, the rebuild chain still runs from its
// graph (a conditional body may hold no event records) and the force launch
// and the timing events are issued around it.

__global__ void rebuild_cond_kernel(cudaGraphConditionalHandle c, DevStatus *ds) {
    const unsigned run = (ds->status == 0 && ds->rebuild != 0) ? 1u : 0u;
    if (run) ds->cond_runs += 1;
    cudaGraphSetConditional(c, run);
}

void drop_graphs(md_system *h) {
    for (int b = 0; b < 2; ++b) {
        if (h->gexec[b]) {
            cudaGraphExecDestroy(h->gexec[b]);
            h->gexec[b] = nullptr;
        }
        if (h->gexec_rb[b]) {
            cudaGraphExecDestroy(h->gexec_rb[b]);
            h->gexec_rb[b] = nullptr;
        }
    }
}

// Captures, for the current parity, [condition kernel] -> [IF: rebuild chain]
// and, with with_forces, -> [fused force + kick + drift].  On any failure the
// handle falls back to plain launches (graphs_ok = false).
md_status capture_step_graph(md_system *h, bool with_forces, cudaGraphExec_t *out,
                             long long *uncond_launches) {
    const long long l0 = h->launches;
    const bool timing = h->timing;
    h->timing = false;  // no event records inside a graph
    md_status st = MD_OK;
    cudaGraph_t graph = nullptr;
    cudaGraphConditionalHandle cond = 0;
    cudaGraphNode_t knode = nullptr, inode = nullptr;
    cudaGraphNodeParams cp = {};
    // one stream capture into graph g after the nodes dep[0..ndep)
    auto capture = [&](cudaGraph_t g, const cudaGraphNode_t *dep, size_t ndep,
                       const auto &body) -> cudaError_t {
        cudaError_t r = cudaStreamBeginCaptureToGraph(h->stream, g, dep, nullptr, ndep,
                                                      cudaStreamCaptureModeThreadLocal);
        if (r != cudaSuccess) return r;
        const md_status sb = body();
        cudaGraph_t gg = g;
        r = cudaStreamEndCapture(h->stream, &gg);
        if (sb != MD_OK) {
            st = sb;
            return cudaErrorUnknown;
        }
        return r;
    };
    cudaError_t e = cudaGraphCreate(&graph, 0);
    if (e == cudaSuccess)
        e = cudaGraphConditionalHandleCreate(&cond, graph, 0, cudaGraphCondAssignDefault);
    if (e == cudaSuccess)
        e = capture(graph, nullptr, 0, [&]() -> md_status {
            rebuild_cond_kernel<<<1, 1, 0, h->stream>>>(cond, h->ds);
            h->launches += 1;
            return cudaGetLastError() == cudaSuccess ? MD_OK : MD_ERR_CUDA;
        });
    if (e == cudaSuccess) {
        size_t nn = 1;
        e = cudaGraphGetNodes(graph, &knode, &nn);
        if (e == cudaSuccess && nn != 1) e = cudaErrorUnknown;
    }
    if (e == cudaSuccess) {
        cp.type = cudaGraphNodeTypeConditional;
        cp.conditional.handle = cond;
        cp.conditional.type = cudaGraphCondTypeIf;
        cp.conditional.size = 1;
        e = cudaGraphAddNode(&inode, graph, &knode, nullptr, 1, &cp);
    }
    const long long lb = h->launches;
    if (e == cudaSuccess)
        e = capture(cp.conditional.phGraph_out[0], nullptr, 0,
                    [&]() -> md_status { return enqueue_rebuild(h, true); });
    h->body_launches = h->launches - lb;
    h->launches = lb;  // the body's launches are counted when it runs
    if (e == cudaSuccess && with_forces)
        e = capture(graph, &inode, 1,
                    [&]() -> md_status { return enqueue_forces(h, FM_FUSED_FULL, false, false); });
    if (e == cudaSuccess) e = cudaGraphInstantiate(out, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    *uncond_launches = h->launches - l0;
    h->launches = l0;
    h->timing = timing;
    if (st != MD_OK) return st;
    if (e != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        h->graphs_ok = false;  // fall back to plain launches for this handle
    }
    return MD_OK;
}

bool graphs_usable(const md_system *h) { return h->graphs_ok && h->stream != nullptr; }

// The gated rebuild chain of one step: from the parity's conditional graph
// when graphs work, else as plain gated launches.
md_status enqueue_rebuild_step(md_system *h) {
    const int par = h->cur;
    if (graphs_usable(h)) {
        long long nl = 0;
        if (!h->gexec_rb[par]) {
            md_status st = capture_step_graph(h, false, &h->gexec_rb[par], &nl);
            if (st != MD_OK) return st;
        }
        if (h->gexec_rb[par]) {
            MD_CK(cudaGraphLaunch(h->gexec_rb[par], h->stream));
            h->launches += 1;
            MD_CK(mark(h, K_REBUILD));
            return MD_OK;
        }
    }
    return enqueue_rebuild(h, true);
}

// One step between the first and the last of an md_step call (parity h->cur).
md_status enqueue_full_step(md_system *h) {
    const int par = h->cur;
    if (graphs_usable(h) && !h->timing) {
        if (!h->gexec[par]) {
            md_status st = capture_step_graph(h, true, &h->gexec[par], &h->graph_launches[par]);
            if (st != MD_OK) return st;
        }
        if (h->gexec[par]) {
            MD_CK(cudaGraphLaunch(h->gexec[par], h->stream));
            h->launches += h->graph_launches[par];
            return MD_OK;
        }
    }
    md_status st = enqueue_rebuild_step(h);
    if (st != MD_OK) return st;
    return enqueue_forces(h, FM_FUSED_FULL, false, false);
}

}  // namespace

void mdg::set_thread_error(const std::string &msg) { g_thread_error = msg; }

extern "C" {

// Shared by md_create (one box) and md_create_batch (R boxes, atoms and
// positions concatenated box after box).
// EAM tables, checked and converted for the kernels.
static md_status eam_table(const md_params *p, const md_eam *e, EamTab *t, std::string *why) {
    auto bad = [&](const char *m) { *why = m; return MD_ERR_INVALID; };
    if (!e) return bad("MD_POT_EAM needs md_create_eam");
    if (e->n_phi < 1 || e->n_phi > kEamMaxKnots || e->n_psi < 1 || e->n_psi > kEamMaxKnots)
        return bad("knot counts must be in [1, 16]");
    if (!std::isfinite(e->F_sqrt) || !std::isfinite(e->F_quad))
        return bad("F_sqrt and F_quad must be finite");
    *t = EamTab{};
    t->nphi = e->n_phi;
    t->npsi = e->n_psi;
    for (int k = 0; k < kEamMaxKnots; ++k) {
        const bool ip = k < e->n_phi, iq = k < e->n_psi;
        if ((ip && !(e->phi_r[k] > 0 && e->phi_r[k] <= p->rc && std::isfinite(e->phi_a[k]))) ||
            (iq && !(e->psi_r[k] > 0 && e->psi_r[k] <= p->rc && std::isfinite(e->psi_a[k]))))
            return bad("every knot must lie in (0, rc] with a finite coefficient");
        t->prd[k] = ip ? e->phi_r[k] : 0.0;
        t->pad[k] = ip ? e->phi_a[k] : 0.0;
        t->qrd[k] = iq ? e->psi_r[k] : 0.0;
        t->qad[k] = iq ? e->psi_a[k] : 0.0;
        t->pr[k] = (float)t->prd[k];
        t->pa[k] = (float)t->pad[k];
        t->qr[k] = (float)t->qrd[k];
        t->qa[k] = (float)t->qad[k];
    }
    t->A = e->F_sqrt;
    t->B = e->F_quad;
    return MD_OK;
}

// Species tables of a multi-element Lennard-Jones system, checked and
// converted for the kernels (species of every atom checked on the host).
static md_status type_tables(const md_params *p, const md_lj_types *t, const int32_t *type_dev,
                             int64_t n, TypeTab *tab, std::vector<int32_t> *types,
                             std::string *why) {
    auto bad = [&](const std::string &m) { *why = m; return MD_ERR_INVALID; };
    if (!t || !type_dev) return bad("null species table or species array");
    if (p->potential != MD_POT_LJ) return bad("species tables are for Lennard-Jones");
    const int nt = t->ntypes;
    if (nt < 1 || nt > kMaxTypes) return bad("ntypes must be in [1, 4]");
    *tab = TypeTab{};
    const double rc2 = p->rc * p->rc;
    for (int a = 0; a < nt; ++a) {
        if (!(t->mass[a] > 0) || !std::isfinite(t->mass[a])) return bad("masses must be > 0");
        for (int b = 0; b < nt; ++b) {
            const double e = t->eps[a * nt + b], sg = t->sigma[a * nt + b];
            if (!(e > 0) || !(sg > 0) || !std::isfinite(e + sg))
                return bad("eps and sigma must be > 0");
            if (e != t->eps[b * nt + a] || sg != t->sigma[b * nt + a])
                return bad("eps and sigma must be symmetric");
            const double s2 = sg * sg, sr6 = std::pow(s2 / rc2, 3);
            const int k = a * nt + b;
            tab->e48d[k] = 48 * e;
            tab->e4d[k] = 4 * e;
            tab->s2d[k] = s2;
            tab->shd[k] = 4 * e * (sr6 * sr6 - sr6);
            tab->e48[k] = (float)tab->e48d[k];
            tab->e4[k] = (float)tab->e4d[k];
            tab->s2[k] = (float)s2;
            tab->sh[k] = (float)tab->shd[k];
        }
    }
    types->resize((size_t)n);
    if (cudaMemcpy(types->data(), type_dev, (size_t)n * sizeof(int32_t), cudaMemcpyDeviceToHost) !=
        cudaSuccess)
        return bad("could not read the species array");
    for (int32_t v : *types)
        if (v < 0 || v >= nt) return bad("a species lies outside [0, ntypes)");
    return MD_OK;
}

static md_status create_impl(md_system **out, const md_params *p, int R, const int64_t *n_each,
                             const double *boxes, const double *pos_dev, const double *vel_dev,
                             void *cuda_stream, const char *who, const md_eam *eam = nullptr,
                             const md_lj_types *ltypes = nullptr,
                             const int32_t *type_dev = nullptr) {
    md_system *h = nullptr;
    const std::string W(who);
    if (!out || !p || !boxes || !pos_dev || !n_each || R < 1)
        return fail(nullptr, MD_ERR_INVALID, W + ": null argument");
    *out = nullptr;
    if (R > 65535) return fail(nullptr, MD_ERR_INVALID, W + ": at most 65535 replicas");
    int64_t n = 0;
    std::string why;
    for (int r = 0; r < R; ++r) {
        if (check_params(p, n_each[r], boxes + 3 * r, &why) != MD_OK)
            return fail(nullptr, MD_ERR_INVALID,
                        W + (R > 1 ? ": replica " + std::to_string(r) + ": " : ": ") + why);
        n += n_each[r];
    }
    if (n >= kMaxAtoms) return fail(nullptr, MD_ERR_INVALID, W + ": too many atoms in total");
    EamTab eam_t{};
    if (p->potential == MD_POT_EAM) {
        if (eam_table(p, eam, &eam_t, &why) != MD_OK)
            return fail(nullptr, MD_ERR_INVALID, W + ": " + why);
        if ((p->force_variant != MD_FORCE_FULL && p->force_variant != MD_FORCE_PAIRED) ||
            p->scheduler != MD_SCHED_GRID)
            return fail(nullptr, MD_ERR_INVALID,
                        W + ": the embedded-atom potential runs full lists or two atoms per "
                            "thread under MD_SCHED_GRID");
    } else if (eam) {
        return fail(nullptr, MD_ERR_INVALID, W + ": an EAM table needs MD_POT_EAM");
    }
    TypeTab type_t{};
    std::vector<int32_t> types_h;
    if (ltypes) {
        if (type_tables(p, ltypes, type_dev, n, &type_t, &types_h, &why) != MD_OK)
            return fail(nullptr, MD_ERR_INVALID, W + ": " + why);
        if (R != 1 || (p->force_variant != MD_FORCE_FULL && p->force_variant != MD_FORCE_PAIRED) ||
            p->scheduler != MD_SCHED_GRID)
            return fail(nullptr, MD_ERR_INVALID,
                        W + ": multi-element systems run one box, full lists or two atoms per "
                            "thread, under MD_SCHED_GRID");
    }
    if (p->force_variant == MD_FORCE_CLUSTER &&
        (R != 1 || p->scheduler != MD_SCHED_GRID || ltypes || n >= ((int64_t)1 << 25)))
        return fail(nullptr, MD_ERR_INVALID,
                    W + ": the cluster-pair list runs one one-species box under MD_SCHED_GRID, "
                        "n < 2^25");
    if (p->force_variant != MD_FORCE_FULL && p->force_variant != MD_FORCE_PAIRED &&
        p->potential != MD_POT_LJ)
        return fail(nullptr, MD_ERR_INVALID,
                    W + ": half lists and cluster pairs are built for Lennard-Jones only");
    if ((p->force_variant == MD_FORCE_CLUSTER || p->force_variant == MD_FORCE_PAIRED) &&
        p->precision != MD_MIXED)
        return fail(nullptr, MD_ERR_INVALID,
                    W + ": the cluster and two-atom layouts are built for the mixed path");
    if (R > 1 && (p->potential != MD_POT_LJ || p->precision != MD_MIXED ||
                  (p->force_variant == MD_FORCE_FULL
                       ? (p->scheduler != MD_SCHED_GRID && p->scheduler != MD_SCHED_DYNAMIC)
                       : (p->force_variant != MD_FORCE_PAIRED || p->scheduler != MD_SCHED_GRID))))
        return fail(nullptr, MD_ERR_INVALID,
                    W + ": batches run mixed-precision Lennard-Jones with full lists under "
                        "MD_SCHED_GRID or MD_SCHED_DYNAMIC, or two atoms per thread under "
                        "MD_SCHED_GRID");
    h = new (std::nothrow) md_system();
    if (!h) return fail(nullptr, MD_ERR_OOM, W + ": host allocation failed");
    h->p = *p;
    h->eam = eam_t;
    h->types = type_t;
    h->n = n;
    h->R = R;
    h->stream = (cudaStream_t)cuda_stream;
    h->r_list = p->rc + p->skin;
    h->rl2 = h->r_list * h->r_list;
    h->list_lo = (float)(h->rl2 * (1.0 - 1.0 / 16384.0));
    h->list_hi = (float)(h->rl2 * (1.0 + 1.0 / 16384.0));
    int cells_total = 0;
    h->atom_off_h.assign(1, 0);
    for (int r = 0; r < R; ++r) {
        Grid g{};
        int nc[3];
        for (int d = 0; d < 3; ++d) {
            nc[d] = (int)std::floor(boxes[3 * r + d] / h->r_list);
            g.L[d] = boxes[3 * r + d];
            g.w[d] = boxes[3 * r + d] / nc[d];
            g.inv_w[d] = (double)nc[d] / boxes[3 * r + d];
            g.wf[d] = (float)g.w[d];
            g.inv_wf[d] = (float)g.inv_w[d];
        }
        g.nx = nc[0]; g.ny = nc[1]; g.nz = nc[2];
        g.ncells = nc[0] * nc[1] * nc[2];
        {
            // 2^e <= min(w) < 2^(e+1): its high word bounds offsets below a cell width
            int ex = 0;
            std::frexp(std::min(g.w[0], std::min(g.w[1], g.w[2])), &ex);
            const int e = std::max(-1022, std::min(ex - 1, 1023));
            g.wsmall_hi = (1023 + e) << 20;
        }
        g.cell0 = cells_total;
        cells_total += g.ncells;
        h->grids_h.push_back(g);
        h->atom_off_h.push_back(h->atom_off_h.back() + n_each[r]);
    }
    // h->g: the first box, with the cell count of the whole system
    h->g = h->grids_h[0];
    h->g.ncells = cells_total;
    h->g.cell0 = 0;
    ForceConsts &fc = h->fc;
    const double s2 = p->sigma * p->sigma, rc2 = p->rc * p->rc;
    const double sr6 = std::pow(s2 / rc2, 3);
    fc.rc2 = rc2; fc.sig2 = s2; fc.eps4 = 4 * p->eps; fc.eps48 = 48 * p->eps;
    fc.shift = 4 * p->eps * (sr6 * sr6 - sr6);
    fc.rc2f = (float)rc2; fc.sig2f = (float)s2; fc.eps4f = (float)fc.eps4;
    fc.eps48f = (float)fc.eps48; fc.shiftf = (float)fc.shift;
    fc.sc_a = p->sigma; fc.sc_eps = p->eps; fc.sc_ec = p->eps * p->c;
    fc.sc_af = (float)p->sigma; fc.sc_epsf = (float)p->eps; fc.sc_ecf = (float)(p->eps * p->c);
    fc.sc_n = (int)p->n_exp; fc.sc_m = (int)p->m_exp;
    fc.dt = p->dt; fc.inv_m = 1.0 / p->mass;
    fc.ntypes = ltypes ? ltypes->ntypes : 0;
    for (int t = 0; t < kMaxTypes; ++t) {
        const double m = (ltypes && t < ltypes->ntypes) ? ltypes->mass[t] : p->mass;
        fc.t_inv_m[t] = 1.0 / m;
        h->types_mass[t] = m;
    }
    fc.half_skin2f = (float)(0.25 * p->skin * p->skin);

    const size_t N = (size_t)n, C = (size_t)cells_total;
    const size_t scan_len = std::max(N, C + 1) / (kBlock * 8) + 4;
    cudaError_t e = cudaSuccess;
    auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
    // xq holds one more entry: the far dummy position of the slot lists' padding
    for (int b = 0; b < 2; ++b) { A(dalloc(&h->xr64[b], N)); A(dalloc(&h->xq[b], N + 1)); }
    A(dalloc(&h->xq_build, N)); A(dalloc(&h->xabs, N)); A(dalloc(&h->v, 3 * N));
    A(dalloc(&h->f, 3 * N)); A(dalloc(&h->e_atom, N)); A(dalloc(&h->orig, N));
    A(dalloc(&h->cell, N)); A(dalloc(&h->cell_start, C + 1)); A(dalloc(&h->cell_count, C));
    A(dalloc(&h->new_cell, N)); A(dalloc(&h->slot, N)); A(dalloc(&h->src, N));
    A(dalloc(&h->key, N)); A(dalloc(&h->scan_bsum, scan_len)); A(dalloc(&h->tmp_abs, N));
    A(dalloc(&h->tmp_v, N)); A(dalloc(&h->ncount, N));
    size_t ctab_len = 0;
    for (const Grid &g : h->grids_h) ctab_len += (size_t)g.nx + g.ny + g.nz;
    A(dalloc(&h->grids, (size_t)R)); A(dalloc(&h->ctab, ctab_len));
    A(dalloc(&h->atom_off, (size_t)R + 1));
    A(dalloc(&h->rep_pe, (size_t)R)); A(dalloc(&h->rep_ke, (size_t)R));
    if (R > 1) {
        A(dalloc(&h->rep, N));
        A(dalloc(&h->shifts32, (size_t)R * kStencil));
    }
    if (p->potential == MD_POT_SC || p->potential == MD_POT_EAM) {
        A(dalloc(&h->rho, N)); A(dalloc(&h->dF32, N)); A(dalloc(&h->dF64, N));
        // one more entry: the far dummy of the slot lists' padding
        if (p->precision == MD_MIXED) A(dalloc(&h->xqf, N + 1));
    }
    h->nblocks_n = nblocks(n);
    A(dalloc(&h->partials, (size_t)h->nblocks_n + 1)); A(dalloc(&h->red_out, 4));
    A(dalloc(&h->ds, 1));
    if (ltypes) {
        A(dalloc(&h->type_orig, N));
        if (e == cudaSuccess)
            e = cudaMemcpy(h->type_orig, types_h.data(), N * sizeof(int32_t),
                           cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->ds_host, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMallocHost((void **)&h->red_host, 4 * sizeof(double));
    if (e != cudaSuccess) {
        md_status st = (e == cudaErrorMemoryAllocation) ? MD_ERR_OOM : MD_ERR_CUDA;
        std::string m = W + ": allocation failed: " + cudaGetErrorString(e);
        cudaGetLastError();
        free_all(h);
        delete h;
        return fail(nullptr, st, m);
    }
    md_status st = MD_OK;
    auto step = [&](cudaError_t r, const char *what) {
        if (st == MD_OK && r != cudaSuccess)
            st = fail(h, MD_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(r));
    };
    std::vector<float4> sh;
    if (R > 1) {
        for (int r = 0; r < R; ++r)
            for (int s = 0; s < kStencil; ++s) {
                const Grid &g = h->grids_h[r];
                const int dx = s % 3 - 1, dy = (s / 3) % 3 - 1, dz = s / 9 - 1;
                sh.push_back(make_float4((float)(dx * g.w[0]), (float)(dy * g.w[1]),
                                         (float)(dz * g.w[2]), 0.f));
            }
        step(cudaMemcpyAsync(h->shifts32, sh.data(), sh.size() * sizeof(float4),
                             cudaMemcpyHostToDevice, h->stream), "copy shifts");
    }
    // cell centres (c + 0.5) w of every box, and each box's pointer into them
    std::vector<double> ctab;
    ctab.reserve(ctab_len);
    for (Grid &g : h->grids_h) {
        g.ctab = h->ctab + ctab.size();
        const int nd[3] = {g.nx, g.ny, g.nz};
        for (int d = 0; d < 3; ++d)
            for (int c = 0; c < nd[d]; ++c) ctab.push_back(((double)c + 0.5) * g.w[d]);
    }
    h->g.ctab = h->grids_h[0].ctab;
    step(cudaMemcpyAsync(h->ctab, ctab.data(), ctab.size() * sizeof(double),
                         cudaMemcpyHostToDevice, h->stream), "copy cell centres");
    step(cudaMemcpyAsync(h->grids, h->grids_h.data(), R * sizeof(Grid), cudaMemcpyHostToDevice,
                         h->stream), "copy grids");
    step(cudaMemcpyAsync(h->atom_off, h->atom_off_h.data(), (R + 1) * sizeof(int64_t),
                         cudaMemcpyHostToDevice, h->stream), "copy offsets");
    step(cudaMemsetAsync(h->ds, 0, sizeof(DevStatus), h->stream), "memset status");
    step(cudaMemsetAsync(h->f, 0, 3 * N * sizeof(double), h->stream), "memset f");
    step(cudaMemsetAsync(h->e_atom, 0, N * sizeof(double), h->stream), "memset e");
    if (!vel_dev) step(cudaMemsetAsync(h->v, 0, 3 * N * sizeof(double), h->stream), "memset v");
    step(launch_pair_dummy(h), "dummy position");
    step(launch_load_state(h, pos_dev, vel_dev), "load_state");
    // host arrays above stay alive until the copies finish
    if (st == MD_OK) step(cudaStreamSynchronize(h->stream), "synchronize");
    if (st == MD_OK && p->scheduler != MD_SCHED_GRID) st = ensure_sched(h);
    if (st == MD_OK) st = rebuild_now(h, true);
    if (st == MD_OK) st = forces_now(h, false);
    if (st != MD_OK) {
        g_thread_error = W + ": " + h->last_error;
        free_all(h);
        delete h;
        return st;
    }
    *out = h;
    return MD_OK;
}

md_status md_create(md_system **out, const md_params *p, int64_t n, const double *box3_host,
                    const double *pos_dev, const double *vel_dev, void *cuda_stream) {
    return create_impl(out, p, 1, &n, box3_host, pos_dev, vel_dev, cuda_stream, "md_create");
}

md_status md_create_eam(md_system **out, const md_params *p, const md_eam *eam_host, int64_t n,
                        const double *box3_host, const double *pos_dev, const double *vel_dev,
                        void *cuda_stream) {
    if (!eam_host) return fail(nullptr, MD_ERR_INVALID, "md_create_eam: null table");
    return create_impl(out, p, 1, &n, box3_host, pos_dev, vel_dev, cuda_stream, "md_create_eam",
                       eam_host);
}

md_status md_create_typed(md_system **out, const md_params *p, const md_lj_types *types_host,
                          const int32_t *type_dev, int64_t n, const double *box3_host,
                          const double *pos_dev, const double *vel_dev, void *cuda_stream) {
    if (!types_host || !type_dev)
        return fail(nullptr, MD_ERR_INVALID, "md_create_typed: null species table or array");
    return create_impl(out, p, 1, &n, box3_host, pos_dev, vel_dev, cuda_stream,
                       "md_create_typed", nullptr, types_host, type_dev);
}

md_status md_create_batch(md_system **out, const md_params *p, int32_t n_replicas,
                          const int64_t *n_each_host, const double *box3_each_host,
                          const double *pos_dev, const double *vel_dev, void *cuda_stream) {
    return create_impl(out, p, n_replicas, n_each_host, box3_each_host, pos_dev, vel_dev,
                       cuda_stream, "md_create_batch");
}

md_status md_energy_batch(md_system *h, double *ke_host, double *pe_host) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_energy_batch: null handle");
    if (h->fc.ntypes > 0) return md_energy(h, ke_host, pe_host);  // one box, species masses
    MD_CK(cudaMemsetAsync(&h->ds->pairs_cut, 0, sizeof(unsigned long long), h->stream));
    md_status st = forces_now(h, true);
    if (st != MD_OK) return st;
    MD_CK(launch_replica_energy(h));
    h->launches += 1;
    if (ke_host)
        MD_CK(cudaMemcpyAsync(ke_host, h->rep_ke, h->R * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
    if (pe_host)
        MD_CK(cudaMemcpyAsync(pe_host, h->rep_pe, h->R * sizeof(double), cudaMemcpyDeviceToHost,
                              h->stream));
    MD_CK(cudaStreamSynchronize(h->stream));
    return MD_OK;
}

md_status md_bin_cells(md_system *h) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_bin_cells: null handle");
    MD_CK(launch_bin(h, false));
    MD_CK(launch_set_rebuild(h));  // list entries now refer to the old order
    h->list_valid = false;
    h->forces_valid = false;
    return MD_OK;
}

md_status md_build_neighbors(md_system *h) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_build_neighbors: null handle");
    return rebuild_now(h, false);
}

md_status md_forces(md_system *h) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_forces: null handle");
    return forces_now(h, false);
}

md_status md_step(md_system *h, int64_t nsteps) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_step: null handle");
    if (nsteps < 0) return fail(h, MD_ERR_INVALID, "md_step: nsteps must be >= 0");
    if (nsteps == 0) return MD_OK;
    if (h->steps_total + nsteps >= (int64_t)1 << 31)
        return fail(h, MD_ERR_INVALID, "md_step: step counter would overflow");
    md_status st;
    if (!h->forces_valid) {
        st = forces_now(h, false);
        if (st != MD_OK) return st;
    }
    const int64_t base = h->steps_total;
    const int c0 = h->cur;
    MD_CK(mark(h, -1));
    begin_steps_kernel<<<1, 1, 0, h->stream>>>(h->ds, (int)base);
    MD_CK(cudaGetLastError());
    MD_CK(launch_kick_drift(h));
    h->launches += 2;
    MD_CK(mark(h, K_INTEGRATE));
    h->forces_valid = false;
    int64_t sr = 1;
    // under timing, the first event of every step (its rebuild mark), so that
    // the launches a list overflow turns into no-ops are not counted
    std::vector<size_t> ev_at;
    if (h->timing) ev_at.assign((size_t)nsteps + 1, 0);
    for (int attempt = 0; attempt < 64; ++attempt) {
        for (int64_t s = sr; s <= nsteps; ++s) {
            h->steps_total = base + s;
            h->cur = c0 ^ (int)((s - 1) & 1);
            if (h->timing) ev_at[s] = h->ev_used;
            if (s < nsteps) {
                st = enqueue_full_step(h);
                if (st != MD_OK) return st;
                continue;
            }
            st = enqueue_rebuild_step(h);
            if (st != MD_OK) return st;
            st = enqueue_forces(h, FM_FUSED_HALF, false, true);
            if (st != MD_OK) return st;
        }
        h->cur = c0 ^ (int)((nsteps - 1) & 1);
        st = read_status(h);
        if (st != MD_OK) return st;
        const int dst = h->ds_host->status;
        if (h->timing) {
            // an overflow in the rebuild before step S stops every later kernel:
            // keep the intervals up to that rebuild, drop the no-op launches
            const int64_t S = (int64_t)h->ds_host->steps_done - base + 1;
            harvest(h, (dst == MD_ERR_LIST_OVERFLOW && S >= 1 && S <= nsteps) ? ev_at[S] + 1
                                                                               : SIZE_MAX);
        }
        if (dst == 0) {
            h->steps_total = base + nsteps;
            h->forces_valid = true;
            h->list_valid = true;
            return MD_OK;
        }
        if (dst != MD_ERR_LIST_OVERFLOW) {
            h->steps_total = h->ds_host->steps_done;
            return fail(h, (md_status)dst, "md_step: device error at step " +
                                               std::to_string(h->ds_host->steps_done + 1));
        }
        // The rebuild before step S overflowed after binning it; grow the list,
        // rebuild it for the same positions and continue with step S.
        const int64_t S = (int64_t)h->ds_host->steps_done - base + 1;
        if (S < 1 || S > nsteps) return fail(h, MD_ERR_STATE, "md_step: inconsistent step counter");
        h->cur = c0 ^ (int)((S - 1) & 1);
        h->steps_total = base + S;
        st = clear_status(h);
        if (st != MD_OK) return st;
        if (h->p.max_neighbors > 0)
            return fail(h, MD_ERR_LIST_OVERFLOW, "md_step: neighbour count exceeds max_neighbors");
        MD_CK(mark(h, -1));  // the repair is timed as one more rebuild
        if (h->p.force_variant == MD_FORCE_PAIRED) {
            st = pair_rebuild_now(h);
            if (st != MD_OK) return st;
        } else {
            MD_CK(alloc_list(h, cap_for(h->ds_host->max_count)));
            MD_CK(launch_build_list(h, true, false));
        }
        if (h->ov_on) MD_CK(launch_overlap_index(h, false));
        if (h->p.force_variant == MD_FORCE_CLUSTER) MD_CK(launch_cluster_build(h, false));
        st = enqueue_sched_prep(h, false);
        if (st != MD_OK) return st;
        MD_CK(launch_finish_rebuild(h, false));
        MD_CK(mark(h, K_REBUILD));
        sr = S;
        // re-enqueue steps S..nsteps; the loop's first rebuild is gated off
        for (int64_t s = sr; s <= nsteps; ++s) {
            h->steps_total = base + s;
            h->cur = c0 ^ (int)((s - 1) & 1);
            if (h->timing) ev_at[s] = h->ev_used;
            if (s > sr) {
                st = enqueue_rebuild(h, true);
                if (st != MD_OK) return st;
            }
            const int mode = (s < nsteps) ? FM_FUSED_FULL : FM_FUSED_HALF;
            st = enqueue_forces(h, mode, false, s == nsteps);
            if (st != MD_OK) return st;
        }
        sr = nsteps + 1;  // everything is enqueued; the outer loop only checks status
    }
    return fail(h, MD_ERR_LIST_OVERFLOW, "md_step: list overflow could not be repaired");
}

md_status md_energy(md_system *h, double *ke_host, double *pe_host) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_energy: null handle");
    MD_CK(cudaMemsetAsync(&h->ds->pairs_cut, 0, sizeof(unsigned long long), h->stream));
    md_status st = forces_now(h, true);
    if (st != MD_OK) return st;
    MD_CK(launch_reduce_pe(h));
    MD_CK(launch_reduce_ke(h));
    h->launches += 4;
    MD_CK(cudaMemcpyAsync(h->red_host, h->red_out, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                          h->stream));
    MD_CK(cudaStreamSynchronize(h->stream));
    if (pe_host) *pe_host = h->red_host[0];
    if (ke_host) *ke_host = h->red_host[1];
    return MD_OK;
}

md_status md_get_state(md_system *h, double *pos_dev, double *vel_dev, double *force_dev) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_get_state: null handle");
    if (force_dev && !h->forces_valid) {
        md_status st = forces_now(h, false);
        if (st != MD_OK) return st;
    }
    MD_CK(launch_get_state(h, pos_dev, vel_dev, force_dev));
    return MD_OK;
}

md_status md_set_state(md_system *h, const double *pos_dev, const double *vel_dev) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_set_state: null handle");
    if (!pos_dev && !vel_dev) return MD_OK;
    if (pos_dev && !vel_dev) {
        // keep the current velocities: export them in original order first
        double *tmp = nullptr;
        MD_CK(dalloc(&tmp, 3 * (size_t)h->n));
        cudaError_t e = launch_get_state(h, nullptr, tmp, nullptr);
        if (e == cudaSuccess) e = launch_load_state(h, pos_dev, tmp);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        cudaFree(tmp);
        MD_CK(e);
    } else {
        MD_CK(launch_load_state(h, pos_dev, vel_dev));
    }
    if (pos_dev) {
        h->list_valid = false;
        h->forces_valid = false;
    }
    return MD_OK;
}

md_status md_get_neighbors(md_system *h, int32_t half, int64_t *offsets_dev, int32_t *ids_dev,
                           int64_t cap, int64_t *total_host) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_get_neighbors: null handle");
    if (!offsets_dev || cap < 0) return fail(h, MD_ERR_INVALID, "md_get_neighbors: bad argument");
    if (!half && half_variant(h->p.force_variant))
        return fail(h, MD_ERR_INVALID, "md_get_neighbors: the list is a half list");
    if (!h->list_valid) {
        md_status st = rebuild_now(h, false);
        if (st != MD_OK) return st;
    }
    if (h->p.force_variant == MD_FORCE_PAIRED) {
        md_status st = atom_list_for_export(h);
        if (st != MD_OK) return st;
    }
    if (!h->exp_tmp) MD_CK(dalloc(&h->exp_tmp, (size_t)h->n + 64));
    MD_CK(launch_export_list(h, half ? 1 : 0, offsets_dev, nullptr, h->exp_tmp));
    int32_t total32 = 0;
    const int32_t *rowstart = reinterpret_cast<const int32_t *>(h->exp_tmp) + (h->n + 1);
    MD_CK(cudaMemcpyAsync(&total32, rowstart + h->n, sizeof(int32_t), cudaMemcpyDeviceToHost,
                          h->stream));
    MD_CK(cudaStreamSynchronize(h->stream));
    if (total_host) *total_host = total32;
    if (total32 > cap) return fail(h, MD_ERR_LIST_OVERFLOW, "md_get_neighbors: cap too small");
    if (!ids_dev && total32 > 0) return fail(h, MD_ERR_INVALID, "md_get_neighbors: ids_dev is null");
    MD_CK(launch_export_list(h, half ? 1 : 0, offsets_dev, ids_dev, h->exp_tmp));
    MD_CK(cudaStreamSynchronize(h->stream));
    return MD_OK;
}

md_status md_get_cells(md_system *h, int32_t *cell_of_atom_dev, int64_t *cell_start_dev,
                       int32_t *ncell_host) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_get_cells: null handle");
    MD_CK(launch_export_cells(h, cell_of_atom_dev, cell_start_dev));
    MD_CK(cudaStreamSynchronize(h->stream));
    if (ncell_host) {
        // a batch reports its cells as one line, so that the product sizes cell_start
        ncell_host[0] = h->R > 1 ? h->g.ncells : h->g.nx;
        ncell_host[1] = h->R > 1 ? 1 : h->g.ny;
        ncell_host[2] = h->R > 1 ? 1 : h->g.nz;
    }
    return MD_OK;
}

md_status md_get_density(md_system *h, double *rho_dev, double *dF_dev) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_get_density: null handle");
    if (h->p.potential != MD_POT_SC && h->p.potential != MD_POT_EAM)
        return fail(h, MD_ERR_INVALID, "md_get_density: not many-body");
    if (!h->forces_valid) {
        md_status st = forces_now(h, false);
        if (st != MD_OK) return st;
    }
    if (rho_dev) MD_CK(launch_scatter_orig(h, h->rho, rho_dev));
    if (dF_dev) {
        if (h->p.precision == MD_MIXED) MD_CK(launch_scatter_orig_f32(h, h->dF32, dF_dev));
        else MD_CK(launch_scatter_orig(h, h->dF64, dF_dev));
    }
    return MD_OK;
}

md_status md_get_atom_energy(md_system *h, double *e_dev) {
    if (!h || !e_dev) return fail(h, MD_ERR_INVALID, "md_get_atom_energy: null argument");
    MD_CK(launch_scatter_orig(h, h->e_atom, e_dev));
    return MD_OK;
}

md_status md_set_variant(md_system *h, int32_t force_variant, int32_t scheduler) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_set_variant: null handle");
    if (force_variant < MD_FORCE_FULL || force_variant > MD_FORCE_PAIRED ||
        scheduler < MD_SCHED_GRID || scheduler > MD_SCHED_DYNAMIC)
        return fail(h, MD_ERR_INVALID, "md_set_variant: unknown variant or scheduler");
    if (h->ov_on && (force_variant != MD_FORCE_FULL || scheduler != MD_SCHED_GRID))
        return fail(h, MD_ERR_INVALID,
                    "md_set_variant: split (inner/outer) systems run full lists under "
                    "MD_SCHED_GRID");
    if (h->fc.ntypes > 0 && ((force_variant != MD_FORCE_FULL && force_variant != MD_FORCE_PAIRED) ||
                             scheduler != MD_SCHED_GRID))
        return fail(h, MD_ERR_INVALID,
                    "md_set_variant: multi-element systems run full lists or two atoms per "
                    "thread under MD_SCHED_GRID");
    if (h->p.potential == MD_POT_EAM &&
        ((force_variant != MD_FORCE_FULL && force_variant != MD_FORCE_PAIRED) ||
         scheduler != MD_SCHED_GRID))
        return fail(h, MD_ERR_INVALID,
                    "md_set_variant: the embedded-atom potential runs full lists or two atoms "
                    "per thread under MD_SCHED_GRID");
    if (force_variant != MD_FORCE_FULL && force_variant != MD_FORCE_PAIRED &&
        h->p.potential != MD_POT_LJ)
        return fail(h, MD_ERR_INVALID,
                    "md_set_variant: half lists and cluster pairs are built for Lennard-Jones only");
    if ((force_variant == MD_FORCE_CLUSTER || force_variant == MD_FORCE_PAIRED) &&
        h->p.precision != MD_MIXED)
        return fail(h, MD_ERR_INVALID,
                    "md_set_variant: the cluster and two-atom layouts are built for the mixed path");
    if (h->R > 1 && (force_variant == MD_FORCE_FULL
                         ? (scheduler != MD_SCHED_GRID && scheduler != MD_SCHED_DYNAMIC)
                         : (force_variant != MD_FORCE_PAIRED || scheduler != MD_SCHED_GRID)))
        return fail(h, MD_ERR_INVALID,
                    "md_set_variant: batches run full lists under MD_SCHED_GRID or "
                    "MD_SCHED_DYNAMIC, or two atoms per thread under MD_SCHED_GRID");
    if (force_variant == MD_FORCE_CLUSTER &&
        (scheduler != MD_SCHED_GRID || h->n >= ((int64_t)1 << 25)))
        return fail(h, MD_ERR_INVALID,
                    "md_set_variant: the cluster-pair list runs under MD_SCHED_GRID, n < 2^25");
    // a change between half and full pair sets relists; entering the cluster
    // or the two-atom layout builds its tables and list
    const bool relist = half_variant(force_variant) != half_variant(h->p.force_variant) ||
                        (force_variant == MD_FORCE_CLUSTER && h->p.force_variant != MD_FORCE_CLUSTER) ||
                        ((force_variant == MD_FORCE_PAIRED) != (h->p.force_variant == MD_FORCE_PAIRED));
    drop_graphs(h);  // the captured steps launch the old variant's kernels
    h->p.force_variant = force_variant;
    h->p.scheduler = scheduler;
    md_status st = MD_OK;
    if (scheduler != MD_SCHED_GRID) st = ensure_sched(h);
    if (st != MD_OK) return st;
    sched_shape(h);
    if (relist || !h->list_valid) return rebuild_now(h, true);
    // same list: only the partition of the new scheduler is needed
    return enqueue_sched_prep(h, false);
}

md_status md_set_schedule(md_system *h, int32_t rounds, int32_t tail_percent) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_set_schedule: null handle");
    if (rounds < 0 || rounds > kSchedRounds || tail_percent < -1 || tail_percent > kTailPctMax)
        return fail(h, MD_ERR_INVALID,
                    "md_set_schedule: rounds must be 0..16 and tail_percent -1..80");
    drop_graphs(h);  // the captured steps hold the old partition's shape
    h->sched_rounds_set = rounds;
    h->sched_tail_set = tail_percent >= 0;
    if (h->sched_tail_set) h->sched_tail_pct = tail_percent;
    sched_shape(h);
    if (!h->part_bounds) return MD_OK;  // applied when the scheduler allocates
    if (!h->list_valid) return rebuild_now(h, false);
    return enqueue_sched_prep(h, false);
}

md_status md_set_decomposition(md_system *h, int32_t px, int32_t py, int32_t pz) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_set_decomposition: null handle");
    const int p3[3] = {px, py, pz};
    const int nd[3] = {h->g.nx, h->g.ny, h->g.nz};
    for (int d = 0; d < 3; ++d)
        if (p3[d] < 1 || p3[d] > nd[d])
            return fail(h, MD_ERR_INVALID,
                        "md_set_decomposition: 1 <= domains <= cells along every dimension");
    const bool on = px * py * pz > 1;
    if (on && (h->R > 1 || h->p.potential != MD_POT_LJ || h->p.precision != MD_MIXED ||
               h->p.force_variant != MD_FORCE_FULL || h->p.scheduler != MD_SCHED_GRID ||
               h->fc.ntypes > 0))
        return fail(h, MD_ERR_INVALID,
                    "md_set_decomposition: the inner/outer split runs the mixed-precision "
                    "one-species Lennard-Jones full list of one box under MD_SCHED_GRID");
    drop_graphs(h);  // the captured steps launch the other force path
    h->ov_on = false;
    h->dd[0] = px; h->dd[1] = py; h->dd[2] = pz;
    if (!on) return MD_OK;
    const size_t N = (size_t)h->n, C = (size_t)h->g.ncells;
    if (!h->ov_cell_outer) {
        cudaError_t e = cudaSuccess;
        auto A = [&](cudaError_t r) { if (e == cudaSuccess) e = r; };
        A(dalloc(&h->ov_cell_outer, C)); A(dalloc(&h->ov_flag, N)); A(dalloc(&h->ov_pos, N + 1));
        A(dalloc(&h->ov_bsum, N / (kBlock * 8) + 4)); A(dalloc(&h->ov_gidx, N));
        A(dalloc(&h->ov_bidx, N)); A(dalloc(&h->ov_nb, 1)); A(dalloc(&h->ov_send, N));
        A(dalloc(&h->ov_recv, N));
        A(cudaStreamCreateWithFlags(&h->ov_stream, cudaStreamNonBlocking));
        for (cudaEvent_t &ev : h->ov_ev) A(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        if (e != cudaSuccess)
            return fail(h, e == cudaErrorMemoryAllocation ? MD_ERR_OOM : MD_ERR_CUDA,
                        std::string("md_set_decomposition: ") + cudaGetErrorString(e));
    }
    // per cell: the stencil cells that lie in another domain (domain of cell c
    // along a dimension of n cells cut into p domains: floor(c p / n))
    std::vector<uint32_t> outer(C);
    auto dom = [](int c, int n, int p) { return (int)((int64_t)c * p / n); };
    for (int cz = 0; cz < nd[2]; ++cz)
        for (int cy = 0; cy < nd[1]; ++cy)
            for (int cx = 0; cx < nd[0]; ++cx) {
                uint32_t m = 0;
                const int c3[3] = {cx, cy, cz};
                for (int s = 0; s < kStencil; ++s) {
                    const int o3[3] = {s % 3 - 1, (s / 3) % 3 - 1, s / 9 - 1};
                    bool across = false;
                    for (int d = 0; d < 3; ++d) {
                        const int nb = ((c3[d] + o3[d]) % nd[d] + nd[d]) % nd[d];
                        across |= dom(nb, nd[d], p3[d]) != dom(c3[d], nd[d], p3[d]);
                    }
                    if (across) m |= 1u << s;
                }
                outer[((size_t)cz * nd[1] + cy) * nd[0] + cx] = m;
            }
    MD_CK(cudaMemcpyAsync(h->ov_cell_outer, outer.data(), C * sizeof(uint32_t),
                          cudaMemcpyHostToDevice, h->stream));
    h->ov_on = true;
    if (h->list_valid) MD_CK(launch_overlap_index(h, false));
    MD_CK(cudaStreamSynchronize(h->stream));  // the host table above goes out of scope
    return MD_OK;
}

md_status md_get_cell_costs(md_system *h, float *cycles_dev, int64_t *predicted_dev,
                            int64_t *paircount_dev) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_get_cell_costs: null handle");
    if (!h->part_bounds || h->samp_n <= 0)
        return fail(h, MD_ERR_INVALID, "md_get_cell_costs: run md_cost_model(MD_COST_SAMPLE) first");
    const size_t C = (size_t)h->g.ncells;
    if (cycles_dev)
        MD_CK(cudaMemcpyAsync(cycles_dev, h->cell_cycles, C * sizeof(float),
                              cudaMemcpyDeviceToDevice, h->stream));
    if (paircount_dev) {
        MD_CK(launch_cell_features(h, true, false));
        MD_CK(cudaMemcpyAsync(paircount_dev, h->cell_cost, C * sizeof(int64_t),
                              cudaMemcpyDeviceToDevice, h->stream));
    }
    if (predicted_dev) {
        MD_CK(launch_cell_features(h, false, false));
        MD_CK(launch_predict_costs(h, false));
        MD_CK(cudaMemcpyAsync(predicted_dev, h->cell_cost, C * sizeof(int64_t),
                              cudaMemcpyDeviceToDevice, h->stream));
    }
    MD_CK(cudaStreamSynchronize(h->stream));
    return MD_OK;
}

// Per-CTA cycles of one timed force pass, reduced on the host to max / mean.
md_status cta_imbalance(md_system *h, float *out) {
    std::vector<float> c((size_t)h->sched_ctas);
    MD_CK(cudaMemcpyAsync(c.data(), h->cta_cycles, c.size() * sizeof(float),
                          cudaMemcpyDeviceToHost, h->stream));
    MD_CK(cudaStreamSynchronize(h->stream));
    double mx = 0.0, sum = 0.0;
    for (float v : c) {
        mx = std::max(mx, (double)v);
        sum += v;
    }
    if (out) *out = (float)(sum > 0 ? mx / (sum / c.size()) : 0.0);
    return MD_OK;
}

md_status md_cost_model(md_system *h, int32_t op, float *loss_out) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_cost_model: null handle");
    if (h->p.potential != MD_POT_LJ || h->p.precision != MD_MIXED ||
        (h->p.force_variant != MD_FORCE_FULL && h->p.force_variant != MD_FORCE_PAIRED) ||
        h->R > 1 || h->fc.ntypes > 0)
        return fail(h, MD_ERR_INVALID,
                    "md_cost_model: the cost model drives the persistent mixed-precision "
                    "Lennard-Jones full-list force kernel (per atom or two atoms per thread) "
                    "of a single box");
    md_status st = ensure_sched(h);
    if (st != MD_OK) return st;
    const int kPasses = 3, kIters = 400;
    const float kLr = 3e-3f;
    switch (op) {
        case MD_COST_RESET:
            MD_CK(launch_mlp_init(h->mlp_P, 0x1611000075ull, h->stream));
            MD_CK(cudaMemsetAsync(h->mlp_m, 0, kMlpParams * sizeof(float), h->stream));
            MD_CK(cudaMemsetAsync(h->mlp_v, 0, kMlpParams * sizeof(float), h->stream));
            h->mlp_t = 0;
            MD_CK(cudaStreamSynchronize(h->stream));
            return MD_OK;
        case MD_COST_SAMPLE: {
            // a current list, then kPasses timed force passes under the tile queue
            st = enqueue_rebuild(h, true);
            if (st != MD_OK) return st;
            MD_CK(cudaMemsetAsync(h->cell_cycles, 0, (size_t)h->g.ncells * sizeof(float),
                                  h->stream));
            MD_CK(cudaMemsetAsync(h->cta_cycles, 0, (size_t)h->sched_ctas * sizeof(float),
                                  h->stream));
            for (int r = 0; r < kPasses; ++r) MD_CK(launch_lj_persist(h, FM_STORE, true, true, true));
            MD_CK(launch_cell_features(h, false, false));
            int32_t *cnt_dev = h->samp_flag + 2 * ((size_t)h->g.ncells + 1);
            MD_CK(launch_make_samples(h, kPasses, cnt_dev));
            int32_t cnt = 0;
            MD_CK(cudaMemcpyAsync(&cnt, cnt_dev, sizeof(int32_t), cudaMemcpyDeviceToHost,
                                  h->stream));
            st = read_status(h);
            if (st != MD_OK) return st;
            if (h->ds_host->status != 0)
                return fail(h, (md_status)h->ds_host->status, "md_cost_model: device error");
            h->samp_n = cnt;
            h->forces_valid = true;
            if (loss_out) *loss_out = (float)cnt;
            return MD_OK;
        }
        case MD_COST_TRAIN: {
            if (h->samp_n <= 0) return fail(h, MD_ERR_INVALID, "md_cost_model: no samples");
            for (int it = 0; it < kIters; ++it) {
                MD_CK(launch_mlp_loss_grad(h->samp_X, h->samp_y, h->samp_n, h->mlp_P, h->mlp_G,
                                           h->mlp_loss, h->mlp_scratch, h->stream));
                MD_CK(launch_adam(h->mlp_P, h->mlp_G, h->mlp_m, h->mlp_v, kMlpParams, ++h->mlp_t,
                                  kLr, 0.9f, 0.999f, 1e-8f, h->stream));
            }
            MD_CK(launch_mlp_loss_grad(h->samp_X, h->samp_y, h->samp_n, h->mlp_P, h->mlp_G,
                                       h->mlp_loss, h->mlp_scratch, h->stream));
            float loss = 0.f;
            MD_CK(cudaMemcpyAsync(&loss, h->mlp_loss, sizeof(float), cudaMemcpyDeviceToHost,
                                  h->stream));
            MD_CK(cudaStreamSynchronize(h->stream));
            if (loss_out) *loss_out = loss;
            return MD_OK;
        }
        case MD_COST_PREDICT:
            MD_CK(launch_cell_features(h, false, false));
            MD_CK(launch_predict_costs(h, false));
            MD_CK(launch_partition_cells(h, false));
            MD_CK(cudaStreamSynchronize(h->stream));
            return MD_OK;
        case MD_COST_PROFILE: {
            // one timed force pass with the current scheduler: max / mean CTA cycles
            st = enqueue_rebuild(h, true);
            if (st != MD_OK) return st;
            MD_CK(cudaMemsetAsync(h->cell_cycles, 0, (size_t)h->g.ncells * sizeof(float),
                                  h->stream));
            MD_CK(cudaMemsetAsync(h->cta_cycles, 0, (size_t)h->sched_ctas * sizeof(float),
                                  h->stream));
            for (int r = 0; r < kPasses; ++r)
                MD_CK(launch_lj_persist(h, FM_STORE, true,
                                        h->p.scheduler != MD_SCHED_PAIRCOUNT &&
                                            h->p.scheduler != MD_SCHED_MLP,
                                        true));
            st = read_status(h);
            if (st != MD_OK) return st;
            h->forces_valid = true;
            return cta_imbalance(h, loss_out);
        }
        default:
            return fail(h, MD_ERR_INVALID, "md_cost_model: unknown op");
    }
}

md_status md_stats(md_system *h, char *buf_host, size_t cap) {
    if (!h || !buf_host || cap == 0) return fail(h, MD_ERR_INVALID, "md_stats: bad argument");
    md_status st = read_status(h);
    if (st != MD_OK) return st;
    const DevStatus &d = *h->ds_host;
    std::snprintf(buf_host, cap,
                  "{\"n\": %lld, \"ncell\": [%d, %d, %d], \"cap\": %d, \"builds\": %d, "
                  "\"steps\": %lld, \"max_count\": %d, \"max_cell\": %d, \"status\": %d, "
                  "\"precision\": %d, \"force_variant\": %d, \"scheduler\": %d, "
                  "\"list_entries\": %llu, \"pairs_cut\": %llu, \"cluster_pairs\": %llu, "
                  "\"slot_entries\": %llu, \"slot_max\": %d, \"slots\": %d, \"launches\": %lld, "
                  "\"ms\": {\"rebuild\": %.6f, \"force\": %.6f, \"integrate\": %.6f, "
                  "\"other\": %.6f}, \"count\": {\"rebuild\": %lld, \"force\": %lld, "
                  "\"integrate\": %lld, \"other\": %lld}}",
                  (long long)h->n, h->g.nx, h->g.ny, h->g.nz, h->cap, d.builds,
                  (long long)h->steps_total, d.max_count, d.max_cell, d.status, h->p.precision,
                  h->p.force_variant, h->p.scheduler, d.list_entries, d.pairs_cut,
                  d.cluster_pairs, d.pair_entries, d.pair_max, d.pair_slots,
                  h->launches + d.cond_runs * h->body_launches,
                  h->ms_kind[0], h->ms_kind[1], h->ms_kind[2], h->ms_kind[3], h->n_kind[0],
                  h->n_kind[1], h->n_kind[2], h->n_kind[3]);
    return MD_OK;
}

md_status md_set_timing(md_system *h, int32_t on) {
    if (!h) return fail(nullptr, MD_ERR_INVALID, "md_set_timing: null handle");
    MD_CK(cudaStreamSynchronize(h->stream));
    h->timing = (on != 0);
    h->ev_used = 0;
    for (int k = 0; k < 4; ++k) {
        h->ms_kind[k] = 0.0;
        h->n_kind[k] = 0;
    }
    h->launches = 0;
    // rebuild chains run by conditional graph nodes count from here on
    MD_CK(cudaMemsetAsync(&h->ds->cond_runs, 0, sizeof(long long), h->stream));
    return MD_OK;
}

const char *md_last_error(md_system *h) {
    return h ? h->last_error.c_str() : g_thread_error.c_str();
}

void md_destroy(md_system *h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    else cudaDeviceSynchronize();
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    drop_graphs(h);
    free_all(h);
    delete h;
}

}  // extern "C"
