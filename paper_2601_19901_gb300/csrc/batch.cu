// Batched frames (lfdpr_create_batch ... lfdpr_batch_panel in include/lfdpr.h):
// several (display, mesh) scenes of uneven size rendered and interleaved by
// one CUDA graph. The per-scene stages up to the key clear (Sec. 3.1, 3.3) run
// on concurrent graph branches, one persistent launch splats the point pairs
// of every scene (Sec. 3.2), and per-scene resolve (Eq. 8-9) and interleave
// (Sec. 4) follow on the branches. Each scene runs exactly the kernels and
// arithmetic of lfdpr_render_frame + lfdpr_interleave, so its keys, views and
// panel are bit-identical to rendering it alone; the model matrices come from
// device memory so one captured graph replays every frame.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "objects.h"

using namespace lfdpr;

struct lfdpr_batch {
    int n = 0;
    int device = 0, sm_count = 1;
    std::vector<lfdpr_display*> disp;
    std::vector<lfdpr_mesh*> mesh;
    int max_views = 1;
    lfdpr_batch_config cfg{};
    float* d_models = nullptr;       // [n][12] model rows read by k_setup
    float* h_models = nullptr;       // pinned staging of the same
    cudaEvent_t staged = nullptr;    // the last copy out of h_models has run
    SplatScene* d_scenes = nullptr;  // [n] for the batched splat
    cudaStream_t cap = nullptr;      // the stream the graph is captured on
    std::vector<cudaStream_t> br;    // branch streams
    std::vector<cudaEvent_t> ev;     // fork, fork2, joins
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool stale = true;               // capture again before the next replay
    std::vector<cudaEvent_t> tev;    // timing: [0] the batch starts, [1 + i] scene i's panel is done
    bool replayed = false;           // a graph with the timing events has been launched
    std::vector<lfdpr_batch_config> tried;   // the last autotune's candidates
    std::vector<float> tried_ms;             // and their mean ms per batch
};

namespace {

#define g_err lfdpr::g_last_error

#define CK(call, what)                                      \
    do {                                                    \
        cudaError_t e_ = (call);                            \
        if (e_ != cudaSuccess) return cuda_fail(e_, what);  \
    } while (0)

const int kSlotChoices[] = {1, 2, 3, 4, 6, 8};

int fewest_slots(int views) {
    for (int s : kSlotChoices)
        if (16 * s >= views) return s;
    return 8;
}

bool valid_slots(int s) {
    for (int v : kSlotChoices)
        if (v == s) return true;
    return false;
}

void drop_graph(lfdpr_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->stale = true;
}

void drop_branches(lfdpr_batch* b) {
    for (auto s : b->br) cudaStreamDestroy(s);
    for (auto e : b->ev) cudaEventDestroy(e);
    b->br.clear();
    b->ev.clear();
}

void free_batch(lfdpr_batch* b) {
    if (!b) return;
    drop_graph(b);
    drop_branches(b);
    for (auto e : b->tev)
        if (e) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->staged) cudaEventDestroy(b->staged);
    dev_free(b->d_models);
    host_free(b->h_models);
    dev_free(b->d_scenes);
    delete b;
}

// Record the whole batch on b->cap (which is capturing).
lfdpr_status record_batch(lfdpr_batch* b) {
    const int K = b->cfg.branches;
    cudaStream_t s = b->cap;
    cudaEvent_t fork = b->ev[0], fork2 = b->ev[1];
    // timing events as event-record nodes of the graph (a plain record during
    // capture would only join streams)
    CK(cudaEventRecordWithFlags(b->tev[0], s, cudaEventRecordExternal), "batch: start event");
    CK(cudaEventRecord(fork, s), "batch: fork");
    for (int j = 0; j < K; j++) CK(cudaStreamWaitEvent(b->br[j], fork, 0), "batch: branch wait");
    for (int i = 0; i < b->n; i++) {
        FrameArgs a = frame_args(b->disp[i], b->mesh[i]);
        a.model_dev = b->d_models + 12 * i;
        const lfdpr_status st = record_frame_front(b->disp[i], b->mesh[i], a, b->br[i % K], false);
        if (st != LFDPR_OK) return st;
    }
    for (int j = 0; j < K; j++) {
        CK(cudaEventRecord(b->ev[2 + j], b->br[j]), "batch: join");
        CK(cudaStreamWaitEvent(s, b->ev[2 + j], 0), "batch: join wait");
    }
    CK(launch_splat_batch(b->d_scenes, b->n, b->cfg.splat_slots, b->cfg.splat_blocks_per_sm, b->sm_count, s),
       "launch k_splat_batch");
    CK(cudaEventRecord(fork2, s), "batch: fork");
    for (int j = 0; j < K; j++) CK(cudaStreamWaitEvent(b->br[j], fork2, 0), "batch: branch wait");
    for (int i = 0; i < b->n; i++) {
        const FrameArgs a = frame_args(b->disp[i], b->mesh[i]);
        CK(launch_resolve(a, b->br[i % K]), "launch k_resolve");
        lfdpr_display* d = b->disp[i];
        if ((d->desc.recon == 2 || d->desc.recon == 3) && d->n_samples == 0)
            return fail(LFDPR_EINVAL, "batch: scene %d needs lfdpr_set_recon_samples", i);
        const lfdpr_status sti = record_interleave(b->disp[i], d->panel, b->br[i % K]);
        if (sti != LFDPR_OK) return sti;
        CK(cudaEventRecordWithFlags(b->tev[1 + i], b->br[i % K], cudaEventRecordExternal), "batch: scene event");
    }
    for (int j = 0; j < K; j++) {
        CK(cudaEventRecord(b->ev[2 + K + j], b->br[j]), "batch: join");
        CK(cudaStreamWaitEvent(s, b->ev[2 + K + j], 0), "batch: join wait");
    }
    return LFDPR_OK;
}

lfdpr_status capture(lfdpr_batch* b) {
    drop_graph(b);
    const int K = b->cfg.branches;
    if ((int)b->br.size() != K) {
        drop_branches(b);
        b->br.resize(K, nullptr);
        b->ev.resize(2 + 2 * K, nullptr);
        for (auto& s : b->br) CK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "batch: stream");
        for (auto& e : b->ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "batch: event");
    }
    CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed), "batch: begin capture");
    const lfdpr_status st = record_batch(b);
    cudaGraph_t g = nullptr;
    const cudaError_t e = cudaStreamEndCapture(b->cap, &g);
    if (st != LFDPR_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(e, "batch: end capture");
    }
    b->graph = g;
    CK(cudaGraphInstantiate(&b->exec, b->graph, 0), "batch: instantiate");
    b->stale = false;
    return LFDPR_OK;
}

lfdpr_status check_config(const lfdpr_batch* b, const lfdpr_batch_config& c) {
    if (c.branches < 1 || c.branches > 32) return fail(LFDPR_EINVAL, "batch: branches must be in [1, 32]");
    if (c.splat_blocks_per_sm < 1 || c.splat_blocks_per_sm > 64)
        return fail(LFDPR_EINVAL, "batch: splat_blocks_per_sm must be in [1, 64]");
    if (!valid_slots(c.splat_slots)) return fail(LFDPR_EINVAL, "batch: splat_slots must be 1, 2, 3, 4, 6 or 8");
    (void)b;
    return LFDPR_OK;
}

}  // namespace

extern "C" {

lfdpr_status lfdpr_create_batch(lfdpr_display* const* displays, lfdpr_mesh* const* meshes, int32_t n,
                                lfdpr_batch** out) {
    g_err[0] = 0;
    if (!displays || !meshes || !out) return fail(LFDPR_EINVAL, "create_batch: null argument");
    *out = nullptr;
    if (n < 1 || n > kMaxBatchScenes) return fail(LFDPR_EINVAL, "create_batch: n must be in [1, %d]", kMaxBatchScenes);
    int views = 0, max_views = 1;
    for (int i = 0; i < n; i++) {
        if (!displays[i] || !meshes[i]) return fail(LFDPR_EINVAL, "create_batch: null display or mesh %d", i);
        if (meshes[i]->disp != displays[i])
            return fail(LFDPR_EINVAL, "create_batch: mesh %d was uploaded to another display", i);
        for (int k = 0; k < i; k++)
            if (displays[k] == displays[i]) return fail(LFDPR_EINVAL, "create_batch: display %d repeated", i);
        if (displays[i]->device != displays[0]->device)
            return fail(LFDPR_EINVAL, "create_batch: scenes on different devices");
        views += displays[i]->dc.nr;
        max_views = std::max(max_views, displays[i]->dc.nr);
    }
    if (views > kMaxBatchViews)
        return fail(LFDPR_EINVAL, "create_batch: %d rendered views in all, at most %d", views, kMaxBatchViews);
    lfdpr_batch* b = new (std::nothrow) lfdpr_batch();
    if (!b) return fail(LFDPR_ENOMEM, "host allocation failed");
    b->n = n;
    b->disp.assign(displays, displays + n);
    b->mesh.assign(meshes, meshes + n);
    b->device = displays[0]->device;
    b->sm_count = displays[0]->sm_count;
    b->max_views = max_views;
    b->cfg.branches = std::min(4, n);
    b->cfg.splat_blocks_per_sm = 16;
    b->cfg.splat_slots = fewest_slots(max_views);
    std::vector<SplatScene> sc(n);
    for (int i = 0; i < n; i++) {
        sc[i].dc = displays[i]->dc;
        sc[i].ex = displays[i]->d_ex;
        sc[i].ctr = displays[i]->ctr;
        sc[i].work = displays[i]->work;
        sc[i].rec = meshes[i]->rec;
        sc[i].keys = displays[i]->keys;
    }
    cudaError_t e;
    if ((e = dev_malloc(&b->d_models, sizeof(float) * 12 * n)) != cudaSuccess ||
        (e = host_malloc(&b->h_models, sizeof(float) * 12 * n)) != cudaSuccess ||
        (e = dev_malloc(&b->d_scenes, sizeof(SplatScene) * n)) != cudaSuccess ||
        (e = cudaMemcpy(b->d_scenes, sc.data(), sizeof(SplatScene) * n, cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->staged, cudaEventDisableTiming)) != cudaSuccess ||
        (e = [&] {
            b->tev.assign(n + 1, nullptr);
            for (auto& t : b->tev) {
                const cudaError_t r = cudaEventCreate(&t);
                if (r != cudaSuccess) return r;
            }
            return cudaSuccess;
        }()) != cudaSuccess ||
        (e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "create_batch");
    }
    *out = b;
    return LFDPR_OK;
}

lfdpr_status lfdpr_destroy_batch(lfdpr_batch* batch) {
    g_err[0] = 0;
    if (!batch) return fail(LFDPR_EINVAL, "destroy_batch: null");
    cudaEventSynchronize(batch->staged);
    free_batch(batch);
    return LFDPR_OK;
}

lfdpr_status lfdpr_batch_get_config(const lfdpr_batch* batch, lfdpr_batch_config* out) {
    g_err[0] = 0;
    if (!batch || !out) return fail(LFDPR_EINVAL, "batch_get_config: null argument");
    *out = batch->cfg;
    return LFDPR_OK;
}

lfdpr_status lfdpr_batch_set_config(lfdpr_batch* batch, const lfdpr_batch_config* cfg) {
    g_err[0] = 0;
    if (!batch || !cfg) return fail(LFDPR_EINVAL, "batch_set_config: null argument");
    const lfdpr_status st = check_config(batch, *cfg);
    if (st != LFDPR_OK) return st;
    if (std::memcmp(&batch->cfg, cfg, sizeof *cfg) != 0) {
        batch->cfg = *cfg;
        batch->stale = true;
    }
    return LFDPR_OK;
}

lfdpr_status lfdpr_render_batch(lfdpr_batch* b, const float* models, void* stream) {
    g_err[0] = 0;
    if (!b || !models) return fail(LFDPR_EINVAL, "render_batch: null argument");
    for (int i = 0; i < b->n; i++)
        for (int k = 0; k < 12; k++)
            if (!std::isfinite(models[16 * i + k]))
                return fail(LFDPR_EINVAL, "render_batch: non-finite model matrix of scene %d", i);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    CK(cudaEventSynchronize(b->staged), "render_batch: staging");
    for (int i = 0; i < b->n; i++) std::memcpy(b->h_models + 12 * i, models + 16 * i, sizeof(float) * 12);
    CK(cudaMemcpyAsync(b->d_models, b->h_models, sizeof(float) * 12 * b->n, cudaMemcpyHostToDevice, s),
       "render_batch: models");
    CK(cudaEventRecord(b->staged, s), "render_batch: staging");
    if (b->stale) {
        const lfdpr_status st = capture(b);
        if (st != LFDPR_OK) return st;
    }
    CK(cudaGraphLaunch(b->exec, s), "render_batch: graph launch");
    b->replayed = true;
    for (int i = 0; i < b->n; i++) {
        b->disp[i]->ev_frame = b->disp[i]->ev_interleave = false;
        // set-up, scan, emission, fetch, near-limit records (and the
        // materials' fetch), resolve, (view mips,) interleave
        b->disp[i]->launches += (b->mesh[i]->n_tris ? (b->mesh[i]->mat_tex ? 8 : 7) : 2) + (b->disp[i]->ss_level > 0);
    }
    b->disp[0]->launches += 1;
    return LFDPR_OK;
}

lfdpr_status lfdpr_batch_autotune(lfdpr_batch* b, const float* models, int32_t reps, void* stream,
                                  lfdpr_batch_config* best_out, float* best_ms_out) {
    g_err[0] = 0;
    if (!b || !models || reps < 1) return fail(LFDPR_EINVAL, "batch_autotune: null argument or reps < 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // Candidates: branch counts, persistent-splat grid sizes, and view slots
    // per lane (the fewest that hold the largest view count, and half that
    // where the scenes' view counts make two groups of it fit).
    std::vector<int> ks, gs = {4, 8, 16}, ss;
    for (int k : {1, 2, 4, 8, 16})
        if (k <= b->n) ks.push_back(k);
    ss.push_back(fewest_slots(b->max_views));
    for (int v : kSlotChoices)
        if (2 * v == ss[0]) ss.push_back(v);
    cudaEvent_t t0, t1;
    CK(cudaEventCreate(&t0), "autotune: event");
    CK(cudaEventCreate(&t1), "autotune: event");
    lfdpr_batch_config best = b->cfg;
    float best_ms = INFINITY;
    lfdpr_status st = LFDPR_OK;
    b->tried.clear();
    b->tried_ms.clear();
    for (int k : ks)
        for (int g : gs)
            for (int sl : ss) {
                const lfdpr_batch_config c{k, g, sl};
                if ((st = lfdpr_batch_set_config(b, &c)) != LFDPR_OK) break;
                if ((st = lfdpr_render_batch(b, models, stream)) != LFDPR_OK) break;   // capture + warm-up
                cudaEventRecord(t0, s);
                for (int r = 0; r < reps && st == LFDPR_OK; r++) st = lfdpr_render_batch(b, models, stream);
                if (st != LFDPR_OK) break;
                cudaEventRecord(t1, s);
                float ms = 0.0f;
                cudaError_t e = cudaEventSynchronize(t1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
                if (e != cudaSuccess) {
                    st = cuda_fail(e, "autotune: timing");
                    break;
                }
                ms /= float(reps);
                b->tried.push_back(c);
                b->tried_ms.push_back(ms);
                if (ms < best_ms) {
                    best_ms = ms;
                    best = c;
                }
            }
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    if (st != LFDPR_OK) return st;
    st = lfdpr_batch_set_config(b, &best);
    if (st != LFDPR_OK) return st;
    if (best_out) *best_out = best;
    if (best_ms_out) *best_ms_out = best_ms;
    return LFDPR_OK;
}

lfdpr_status lfdpr_batch_autotune_table(const lfdpr_batch* batch, lfdpr_batch_config* cfgs, float* ms,
                                        int32_t capacity, int32_t* n) {
    g_err[0] = 0;
    if (!batch || !n) return fail(LFDPR_EINVAL, "batch_autotune_table: null argument");
    *n = int32_t(batch->tried.size());
    for (int32_t k = 0; k < *n && k < capacity; k++) {
        if (cfgs) cfgs[k] = batch->tried[k];
        if (ms) ms[k] = batch->tried_ms[k];
    }
    return LFDPR_OK;
}

lfdpr_status lfdpr_batch_scene_ms(const lfdpr_batch* batch, float* ms, int32_t capacity) {
    g_err[0] = 0;
    if (!batch || !ms) return fail(LFDPR_EINVAL, "batch_scene_ms: null argument");
    if (capacity < batch->n) return fail(LFDPR_EINVAL, "batch_scene_ms: capacity %d < %d scenes", capacity, batch->n);
    if (!batch->replayed) return fail(LFDPR_EINVAL, "batch_scene_ms: no batch rendered yet");
    for (int i = 0; i < batch->n; i++) {
        CK(cudaEventSynchronize(batch->tev[1 + i]), "batch_scene_ms: synchronize");
        CK(cudaEventElapsedTime(&ms[i], batch->tev[0], batch->tev[1 + i]), "batch_scene_ms: elapsed");
    }
    return LFDPR_OK;
}

lfdpr_status lfdpr_batch_panel(const lfdpr_batch* batch, int32_t i, const uint8_t** panel) {
    g_err[0] = 0;
    if (!batch || !panel) return fail(LFDPR_EINVAL, "batch_panel: null argument");
    if (i < 0 || i >= batch->n) return fail(LFDPR_EINVAL, "batch_panel: scene %d out of range", i);
    *panel = batch->disp[i]->panel;
    return LFDPR_OK;
}

}  // extern "C"
