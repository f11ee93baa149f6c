// Batched runs (scivr_batch_*): many molecules with different F, trajectory
// counts and step counts.  Trajectories of all molecules are independent
// (Sec. III.B of arXiv:1312.4698), so the plan groups molecules by
// (F, precision) and runs each mixed-precision group as one persistent
// lane-group launch whose CTAs pull (molecule, tile) work items, the
// longest first.  FP64 molecules are launched one by one.  Each molecule's
// spectra follow.  The launch sequence allocates nothing and never
// synchronises, so it can be captured into a CUDA graph.
//
// The CTA shape (warps per CTA) of each group is picked by timing the
// candidates on a short probe of the group's first molecule (64 steps,
// enough trajectories to fill the GPU) and cached per (F, precision,
// device name) in-process and, when SCIVR_TUNE_CACHE names a file, on disk.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "scivr_internal.cuh"

namespace {

using namespace scivr;

struct Group {
    int F = 0, precision = 0, warps = 0;
    std::vector<int> members;          // indices into the plan's items
    PropLaunch *d_items = nullptr;
    int2 *d_work = nullptr;
    int n_work = 0;
    int *d_counter = nullptr;
};

std::mutex g_tune_mu;
std::map<std::string, int> g_tuned;

std::string tune_key(int F, int precision)
{
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp p{};
    cudaGetDeviceProperties(&p, dev);
    std::string name = p.name;
    for (char &c : name)
        if (c == ' ') c = '_';
    return "F" + std::to_string(F) + ":prec" + std::to_string(precision) + ":" + name;
}

void load_tune_file()
{
    const char *path = std::getenv("SCIVR_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    char key[256];
    int w = 0;
    while (std::fscanf(f, "%255s %d", key, &w) == 2) g_tuned[key] = w;
    std::fclose(f);
}

void save_tune_file()
{
    const char *path = std::getenv("SCIVR_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "w");
    if (!f) return;
    for (auto &kv : g_tuned) std::fprintf(f, "%s %d\n", kv.first.c_str(), kv.second);
    std::fclose(f);
}

// Time one candidate CTA shape on a probe copy of launch record L.
cudaError_t time_candidate(const PropLaunch &L, int warps, int n_sm, float *ms)
{
    const int G = mixed_group_lanes(L.args.F);
    const int per_tile = warps * (32 / G);
    PropLaunch P = L;
    P.args.n_steps = std::min(L.args.n_steps, 64);
    P.n_traj = std::min<int64_t>(L.n_traj, (int64_t)n_sm * 4 * per_tile);
    P.amp_ld = P.args.n_steps + 1;
    P.chi_stride = P.n_traj * P.amp_ld;
    P.fin = FinalDev{};
    const int tiles = (int)((P.n_traj + per_tile - 1) / per_tile);
    std::vector<int2> work(tiles);
    for (int i = 0; i < tiles; ++i) work[i] = make_int2(0, i);
    void *mem = nullptr;
    const size_t amp_bytes = sizeof(double2) * (size_t)P.args.n_chi * P.chi_stride;
    const size_t bytes = amp_bytes + P.n_traj + sizeof(PropLaunch) + sizeof(int2) * tiles + 256 * 4;
    cudaError_t e = cudaMalloc(&mem, bytes);
    if (e != cudaSuccess) return e;
    char *b = static_cast<char *>(mem);
    P.amp = reinterpret_cast<double2 *>(b);
    P.good = reinterpret_cast<uint8_t *>(b + amp_bytes);
    size_t off = (amp_bytes + P.n_traj + 255) & ~(size_t)255;
    PropLaunch *d_items = reinterpret_cast<PropLaunch *>(b + off);
    off = (off + sizeof(PropLaunch) + 255) & ~(size_t)255;
    int2 *d_work = reinterpret_cast<int2 *>(b + off);
    off = (off + sizeof(int2) * tiles + 255) & ~(size_t)255;
    int *d_counter = reinterpret_cast<int *>(b + off);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaMemcpy(d_items, &P, sizeof(PropLaunch), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d_work, work.data(), sizeof(int2) * tiles, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float best = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        e = cudaMemset(d_counter, 0, sizeof(int));
        if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
        if (e == cudaSuccess) e = launch_group_batch_mixed(P.args.F, warps, d_items, d_work, tiles, d_counter, n_sm, 0);
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.0f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && rep > 0) best = std::min(best, t);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(mem);
    *ms = best;
    return e;
}

cudaError_t choose_warps(const PropLaunch &L, int precision, int n_sm, int *warps)
{
    int cand[2];
    const int nc = batch_warp_candidates(L.args.F, cand);
    if (nc == 0) return cudaErrorInvalidValue;
    const std::string key = tune_key(L.args.F, precision);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        if (g_tuned.empty()) load_tune_file();
        auto it = g_tuned.find(key);
        if (it != g_tuned.end() && (it->second == cand[0] || it->second == cand[1])) {
            *warps = it->second;
            return cudaSuccess;
        }
    }
    int best_w = cand[0];
    float best_t = 1e30f;
    for (int i = 0; i < nc; ++i) {
        float t = 0.0f;
        cudaError_t e = time_candidate(L, cand[i], n_sm, &t);
        if (e != cudaSuccess) return e;
        if (t < best_t) { best_t = t; best_w = cand[i]; }
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned[key] = best_w;
    save_tune_file();
    *warps = best_w;
    return cudaSuccess;
}

// Relative cost of one trajectory-step at F (the dominant terms of the step's work: the
// quartic Hessian contraction and the monodromy kicks), for ordering work items.
double step_cost(int F)
{
    const double P = F * (F + 1) / 2.0;
    return 6.0 * P * P + 12.0 * F * F * (double)F;
}

// (record, tile) items of the one-launch schedule, the costliest tiles first.
std::vector<int2> multi_work(const std::vector<PropLaunch> &recs)
{
    std::vector<int2> w;
    for (int k = 0; k < (int)recs.size(); ++k) {
        const int per_tile = multi_launch_tile(recs[k].args.F);
        const int tiles = (int)((recs[k].n_traj + per_tile - 1) / per_tile);
        for (int t = 0; t < tiles; ++t) w.push_back(make_int2(k, t));
    }
    std::stable_sort(w.begin(), w.end(), [&](const int2 &a, const int2 &b) {
        const PropLaunch &A = recs[a.x], &Bm = recs[b.x];
        return A.args.n_steps * step_cost(A.args.F) * multi_launch_tile(A.args.F) >
               Bm.args.n_steps * step_cost(Bm.args.F) * multi_launch_tile(Bm.args.F);
    });
    return w;
}

// Time the two schedules of a plan's mixed molecules on a probe (at most 32 steps and
// 2048 trajectories per molecule, amplitudes into a probe buffer): the per-class
// persistent launches one after the other, and the one-launch schedule.  true if the
// one launch is faster.
cudaError_t one_launch_is_faster(const std::vector<PropLaunch> &recs, const std::vector<int> &warps_of_rec,
                                 int n_sm, bool *faster)
{
    std::vector<PropLaunch> P = recs;
    size_t amp_bytes = 0;
    for (auto &L : P) {
        L.args.n_steps = std::min(L.args.n_steps, 32);
        L.n_traj = std::min<int64_t>(L.n_traj, 2048);
        L.amp_ld = L.args.n_steps + 1;
        L.chi_stride = L.n_traj * L.amp_ld;
        L.fin = FinalDev{};
        amp_bytes += ((sizeof(double2) * (size_t)L.args.n_chi * L.chi_stride + (size_t)L.n_traj) + 255) & ~(size_t)255;
    }
    // per-class work lists of the probe
    std::map<int, std::vector<int>> cls;
    for (int k = 0; k < (int)P.size(); ++k) cls[P[k].args.F].push_back(k);
    std::vector<int2> mw = multi_work(P);
    size_t bytes = amp_bytes + sizeof(PropLaunch) * P.size() + sizeof(int2) * (mw.size() + 16) * 2 + 4096 +
                   256 * cls.size();
    for (auto &c : cls) {
        const int per_tile = warps_of_rec[c.second[0]] * (32 / mixed_group_lanes(c.first));
        size_t n = 0;
        for (int k : c.second) n += (P[k].n_traj + per_tile - 1) / per_tile;
        bytes += sizeof(int2) * n + sizeof(PropLaunch) * c.second.size() + 512;
    }
    void *mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, bytes);
    if (e != cudaSuccess) return e;
    char *b = static_cast<char *>(mem);
    for (auto &L : P) {
        L.amp = reinterpret_cast<double2 *>(b);
        b += sizeof(double2) * (size_t)L.args.n_chi * L.chi_stride;
        L.good = reinterpret_cast<uint8_t *>(b);
        b += ((size_t)L.n_traj + 255) & ~(size_t)255;
        b = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(b) + 255) & ~(uintptr_t)255);
    }
    auto put = [&](const void *src, size_t n) -> void * {
        void *dst = b;
        b = reinterpret_cast<char *>((reinterpret_cast<uintptr_t>(b + n) + 255) & ~(uintptr_t)255);
        if (e == cudaSuccess) e = cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
        return dst;
    };
    auto *d_all = static_cast<PropLaunch *>(put(P.data(), sizeof(PropLaunch) * P.size()));
    auto *d_mw = static_cast<int2 *>(put(mw.data(), sizeof(int2) * mw.size()));
    struct ClassProbe { PropLaunch *items; int2 *work; int n_work; int warps; int F; };
    std::vector<ClassProbe> cps;
    for (auto &c : cls) {
        std::vector<PropLaunch> rr;
        for (int k : c.second) rr.push_back(P[k]);
        const int warps = warps_of_rec[c.second[0]];
        const int per_tile = warps * (32 / mixed_group_lanes(c.first));
        std::vector<int2> w;
        for (int k = 0; k < (int)rr.size(); ++k)
            for (int t = 0; t < (int)((rr[k].n_traj + per_tile - 1) / per_tile); ++t) w.push_back(make_int2(k, t));
        ClassProbe cp;
        cp.items = static_cast<PropLaunch *>(put(rr.data(), sizeof(PropLaunch) * rr.size()));
        cp.work = static_cast<int2 *>(put(w.data(), sizeof(int2) * w.size()));
        cp.n_work = (int)w.size();
        cp.warps = warps;
        cp.F = c.first;
        cps.push_back(cp);
    }
    int *counters = reinterpret_cast<int *>(b);   // one per class + one for the one launch
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    float t_class = 1e30f, t_one = 1e30f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        float t = 0.0f;
        e = cudaMemset(counters, 0, sizeof(int) * (cps.size() + 1));
        if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
        for (size_t i = 0; i < cps.size() && e == cudaSuccess; ++i)
            e = launch_group_batch_mixed(cps[i].F, cps[i].warps, cps[i].items, cps[i].work, cps[i].n_work,
                                         counters + i, n_sm, 0);
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && rep > 0) t_class = std::min(t_class, t);
        if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
        if (e == cudaSuccess)
            e = launch_group_batch_multi(d_all, d_mw, (int)mw.size(), counters + cps.size(), n_sm, 0);
        if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && rep > 0) t_one = std::min(t_one, t);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(mem);
    *faster = t_one < t_class;
    return e;
}

}  // namespace

struct scivr_batch_s {
    std::vector<scivr_batch_item> items;
    std::vector<PropLaunch> launches;     // one per item
    std::vector<Group> groups;            // mixed-precision persistent groups
    std::vector<int> fp64_items;          // launched one by one
    int ft_mode = 0;
    int n_sm = 0;
    void *blob = nullptr;                 // work lists, launch records, counters
    void *scratch = nullptr;              // Fourier scratch for the largest molecule
    // one persistent launch for every mixed molecule (when their F classes allow it)
    bool one_launch = false;
    PropLaunch *m_items = nullptr;
    int2 *m_work = nullptr;
    int m_n_work = 0;
    int *m_counter = nullptr;
    void *m_blob = nullptr;
};

extern "C" {

int scivr_batch_create(const scivr_batch_item *items, int32_t n_items, int32_t ft_mode, scivr_batch *out)
{
    if (!items || !out || n_items < 1) return set_error(SCIVR_EINVAL, "scivr_batch_create: need items and n_items >= 1");
    *out = nullptr;
    if (ft_mode != SCIVR_FT_FP64 && ft_mode != SCIVR_FT_CZT64 && ft_tc_digits(ft_mode) == 0)
        return set_error(SCIVR_EUNSUPPORTED, "scivr_batch_create: ft_mode not supported");
    scivr_batch_s *B = new scivr_batch_s;
    B->ft_mode = ft_mode;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&B->n_sm, cudaDevAttrMultiProcessorCount, dev);
    size_t scratch = 0;
    for (int i = 0; i < n_items; ++i) {
        const scivr_batch_item &it = items[i];
        PropLaunch L{};
        int rc = prepare_propagate(it.pes, &it.prm, it.n_traj, it.p0, it.q0, it.amp, it.amp_ld, it.good, nullptr, &L);
        if (rc == SCIVR_OK)
            rc = check_spectrum_args(it.amp, it.amp_ld, it.prm.amp_prec, it.w, it.good, it.n_traj, it.prm.n_steps,
                                     it.prm.dt, it.E_min, it.E_max, it.n_E, ft_mode, it.I_out, "scivr_batch_create");
        if (rc == SCIVR_OK && it.prm.precision == SCIVR_MIXED && it.pes->dev.F > SCIVR_MAX_F)
            rc = set_error(SCIVR_EUNSUPPORTED, "scivr_batch_create: mixed precision is built for F <= 24");
        if (rc == SCIVR_OK && it.pes->dev.kind != SCIVR_PES_POLY)
            rc = set_error(SCIVR_EUNSUPPORTED, "scivr_batch_create: batches take polynomial surfaces");
        if (rc == SCIVR_OK && it.prm.amplitude != SCIVR_AMP_TA)
            rc = set_error(SCIVR_EUNSUPPORTED, "scivr_batch_create: batch spectra are time-averaged (SCIVR_AMP_TA)");
        if (rc == SCIVR_OK && it.pes->dev.mlp.H != 0)
            rc = set_error(SCIVR_EUNSUPPORTED, "scivr_batch_create: potentials with a learned residual run through scivr_propagate");
        if (rc != SCIVR_OK) {
            char msg[600];
            std::snprintf(msg, sizeof msg, "scivr_batch_create: item %d: %s", i, scivr_last_error());
            delete B;
            return set_error(rc, msg);
        }
        B->items.push_back(it);
        B->launches.push_back(L);
        const size_t sb = ft_mode == SCIVR_FT_FP64    ? spectrum_fp64_scratch_bytes(it.n_traj, it.prm.n_steps, it.n_E)
                          : ft_mode == SCIVR_FT_CZT64 ? spectrum_czt_scratch_bytes(it.n_traj, it.prm.n_steps, it.n_E)
                                                      : spectrum_tc_scratch_bytes(ft_mode, it.n_traj, it.prm.n_steps, it.n_E);
        scratch = std::max(scratch, sb);
    }
    // groups
    std::map<int, int> gidx;
    for (int i = 0; i < n_items; ++i) {
        const PropLaunch &L = B->launches[i];
        if (L.args.precision != SCIVR_MIXED) { B->fp64_items.push_back(i); continue; }
        auto f = gidx.find(L.args.F);
        if (f == gidx.end()) {
            gidx[L.args.F] = (int)B->groups.size();
            Group g;
            g.F = L.args.F;
            g.precision = SCIVR_MIXED;
            B->groups.push_back(g);
            f = gidx.find(L.args.F);
        }
        B->groups[f->second].members.push_back(i);
    }
    // autotune each group's CTA shape, then build its work list
    size_t blob_bytes = 0;
    std::vector<std::vector<int2>> works(B->groups.size());
    for (size_t gi = 0; gi < B->groups.size(); ++gi) {
        Group &g = B->groups[gi];
        cudaError_t e = choose_warps(B->launches[g.members[0]], g.precision, B->n_sm, &g.warps);
        if (e != cudaSuccess) {
            delete B;
            return cuda_error(e, "scivr_batch_create: autotune");
        }
        const int G = mixed_group_lanes(g.F);
        const int per_tile = g.warps * (32 / G);
        std::vector<int2> &w = works[gi];
        for (int k = 0; k < (int)g.members.size(); ++k) {
            const PropLaunch &L = B->launches[g.members[k]];
            const int tiles = (int)((L.n_traj + per_tile - 1) / per_tile);
            for (int t = 0; t < tiles; ++t) w.push_back(make_int2(k, t));
        }
        std::stable_sort(w.begin(), w.end(), [&](const int2 &a, const int2 &b) {
            return B->launches[g.members[a.x]].args.n_steps > B->launches[g.members[b.x]].args.n_steps;
        });
        g.n_work = (int)w.size();
        blob_bytes += ((sizeof(PropLaunch) * g.members.size() + 255) & ~(size_t)255) +
                      ((sizeof(int2) * w.size() + 255) & ~(size_t)255) + 256;
    }
    cudaError_t e = cudaSuccess;
    if (blob_bytes) e = cudaMalloc(&B->blob, blob_bytes);
    if (e == cudaSuccess && scratch) e = cudaMalloc(&B->scratch, scratch);
    char *b = static_cast<char *>(B->blob);
    for (size_t gi = 0; gi < B->groups.size() && e == cudaSuccess; ++gi) {
        Group &g = B->groups[gi];
        std::vector<PropLaunch> recs;
        for (int m : g.members) recs.push_back(B->launches[m]);
        g.d_items = reinterpret_cast<PropLaunch *>(b);
        b += (sizeof(PropLaunch) * recs.size() + 255) & ~(size_t)255;
        g.d_work = reinterpret_cast<int2 *>(b);
        b += (sizeof(int2) * works[gi].size() + 255) & ~(size_t)255;
        g.d_counter = reinterpret_cast<int *>(b);
        b += 256;
        e = cudaMemcpy(g.d_items, recs.data(), sizeof(PropLaunch) * recs.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(g.d_work, works[gi].data(), sizeof(int2) * works[gi].size(), cudaMemcpyHostToDevice);
    }
    // one persistent launch for every mixed molecule: built when every mixed class is one the
    // multi-F kernel holds; taken when SCIVR_BATCH_SCHEDULE says "one", or, unless it says
    // "per-class", when the probe finds it faster
    bool multi_ok = B->groups.size() > 1;
    for (const Group &g : B->groups) multi_ok = multi_ok && multi_launch_holds(g.F);
    if (e == cudaSuccess && multi_ok) {
        std::vector<PropLaunch> recs;
        std::vector<int> warps_of_rec;
        for (const Group &g : B->groups)
            for (int m : g.members) {
                recs.push_back(B->launches[m]);
                warps_of_rec.push_back(g.warps);
            }
        const char *sched = std::getenv("SCIVR_BATCH_SCHEDULE");
        bool one = false;
        if (sched && std::strcmp(sched, "one") == 0) one = true;
        else if (!(sched && std::strcmp(sched, "per-class") == 0)) e = one_launch_is_faster(recs, warps_of_rec, B->n_sm, &one);
        if (e == cudaSuccess && one) {
            std::vector<int2> mw = multi_work(recs);
            const size_t nb = ((sizeof(PropLaunch) * recs.size() + 255) & ~(size_t)255) +
                              ((sizeof(int2) * mw.size() + 255) & ~(size_t)255) + 256;
            e = cudaMalloc(&B->m_blob, nb);
            if (e == cudaSuccess) {
                char *mb = static_cast<char *>(B->m_blob);
                B->m_items = reinterpret_cast<PropLaunch *>(mb);
                mb += (sizeof(PropLaunch) * recs.size() + 255) & ~(size_t)255;
                B->m_work = reinterpret_cast<int2 *>(mb);
                mb += (sizeof(int2) * mw.size() + 255) & ~(size_t)255;
                B->m_counter = reinterpret_cast<int *>(mb);
                B->m_n_work = (int)mw.size();
                e = cudaMemcpy(B->m_items, recs.data(), sizeof(PropLaunch) * recs.size(), cudaMemcpyHostToDevice);
                if (e == cudaSuccess)
                    e = cudaMemcpy(B->m_work, mw.data(), sizeof(int2) * mw.size(), cudaMemcpyHostToDevice);
                B->one_launch = e == cudaSuccess;
            }
        }
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        if (B->blob) cudaFree(B->blob);
        if (B->scratch) cudaFree(B->scratch);
        if (B->m_blob) cudaFree(B->m_blob);
        delete B;
        return cuda_error(e, "scivr_batch_create: device setup");
    }
    *out = B;
    clear_error();
    return SCIVR_OK;
}

int scivr_batch_launch(scivr_batch B, void *stream)
{
    if (!B) return set_error(SCIVR_EINVAL, "scivr_batch_launch: NULL plan");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    int launches = 0;
    if (B->one_launch) {
        e = cudaMemsetAsync(B->m_counter, 0, sizeof(int), s);
        if (e == cudaSuccess)
            e = launch_group_batch_multi(B->m_items, B->m_work, B->m_n_work, B->m_counter, B->n_sm, s);
        if (e != cudaSuccess) return cuda_error(e, "scivr_batch_launch: one-launch propagation");
        ++launches;
    }
    for (const Group &g : B->groups) {
        if (B->one_launch) break;
        e = cudaMemsetAsync(g.d_counter, 0, sizeof(int), s);
        if (e == cudaSuccess)
            e = launch_group_batch_mixed(g.F, g.warps, g.d_items, g.d_work, g.n_work, g.d_counter, B->n_sm, s);
        if (e != cudaSuccess) return cuda_error(e, "scivr_batch_launch: propagation group");
        ++launches;
    }
    for (int i : B->fp64_items) {
        int nl = 0;
        e = launch_propagate(B->launches[i], s, &nl);
        launches += nl;
        if (e != cudaSuccess) return cuda_error(e, "scivr_batch_launch: FP64 propagation");
    }
    for (size_t i = 0; i < B->items.size(); ++i) {
        const scivr_batch_item &it = B->items[i];
        for (int x = 0; x < it.prm.n_chi; ++x) {
            const AmpRef amp = AmpRef{it.amp, it.prm.amp_prec == SCIVR_MIXED}.offset((int64_t)x * it.n_traj * it.amp_ld);
            double *I = it.I_out + (int64_t)x * it.n_E;
            int nl = 0;
            if (B->ft_mode == SCIVR_FT_FP64)
                e = launch_spectrum_fp64(amp, it.amp_ld, it.w, it.good, it.n_traj, it.prm.n_steps, it.prm.dt,
                                         it.E_min, it.E_max, it.n_E, I, it.n_good_out, B->scratch, s, &nl);
            else if (B->ft_mode == SCIVR_FT_CZT64)
                e = launch_spectrum_czt(amp, it.amp_ld, it.w, it.good, it.n_traj, it.prm.n_steps, it.prm.dt,
                                        it.E_min, it.E_max, it.n_E, I, it.n_good_out, B->scratch, s, &nl);
            else
                e = launch_spectrum_tc(B->ft_mode, amp, it.amp_ld, it.w, it.good, it.n_traj, it.prm.n_steps,
                                       it.prm.dt, it.E_min, it.E_max, it.n_E, I, it.n_good_out, B->scratch, s, &nl);
            launches += nl;
            if (e != cudaSuccess) return cuda_error(e, "scivr_batch_launch: spectrum");
        }
    }
    count_launches(launches);
    clear_error();
    return SCIVR_OK;
}

int scivr_batch_info(scivr_batch B, int32_t g, int32_t *n_groups, int32_t *F, int32_t *precision, int32_t *warps)
{
    if (!B) return set_error(SCIVR_EINVAL, "scivr_batch_info: NULL plan");
    if (n_groups) *n_groups = (int32_t)B->groups.size();
    if (g >= 0 && g < (int32_t)B->groups.size()) {
        if (F) *F = B->groups[g].F;
        if (precision) *precision = B->groups[g].precision;
        if (warps) *warps = B->groups[g].warps;
    } else if (F || precision || warps) {
        return set_error(SCIVR_EINVAL, "scivr_batch_info: group index out of range");
    }
    clear_error();
    return SCIVR_OK;
}

int scivr_batch_schedule(scivr_batch B, int32_t *one_launch)
{
    if (!B || !one_launch) return set_error(SCIVR_EINVAL, "scivr_batch_schedule: NULL argument");
    *one_launch = B->one_launch ? 1 : 0;
    clear_error();
    return SCIVR_OK;
}

int scivr_batch_destroy(scivr_batch B)
{
    if (!B) { clear_error(); return SCIVR_OK; }
    cudaError_t e = cudaDeviceSynchronize();
    if (B->blob) cudaFree(B->blob);
    if (B->scratch) cudaFree(B->scratch);
    if (B->m_blob) cudaFree(B->m_blob);
    delete B;
    if (e != cudaSuccess) return cuda_error(e, "scivr_batch_destroy: synchronize");
    clear_error();
    return SCIVR_OK;
}

}  // extern "C"
