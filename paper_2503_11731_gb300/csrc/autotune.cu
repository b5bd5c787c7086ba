// autotune.cu -- gsr_autotune: tile shape and staging depth of the rig frame.
//
// The free parameters of the tiled renderer are the screen tile of each
// sensor kind, the number of records staged per step of a tile's walk and
// the lengths in which long tile lists are split (longer chunks waste less
// speculative work, shorter ones shorten the critical path).
// Small tiles shorten each ray's list (fewer evaluations) but duplicate
// more surfel/tile pairs (more sorting); the staging depth trades shared
// memory (occupancy) against barrier and copy overhead.  Neither changes a
// result.  The tuner times whole frames (preprocess + bin_sort +
// render_rig) with CUDA events and descends one coordinate at a time.
#include <cstring>
#include <vector>

#include "gsr_internal.cuh"

namespace gsr {
gsr_status cuda_status(cudaError_t e);
}

namespace {

constexpr int kLid = GSR_AUTOTUNE_LIDARS;

struct Candidate {
    int cam[2];
    int lid[kLid][2];  // LiDAR k's tile (plan order; later LiDARs take the last)
    int bd;
    int sf, sc;    // the plan's split_first, split_chunk (the cameras')
    int lsf, lsc;  // the LiDARs' own (0 = the plan's)
};

bool same(const Candidate& a, const Candidate& b)
{
    for (int k = 0; k < kLid; ++k)
        if (a.lid[k][0] != b.lid[k][0] || a.lid[k][1] != b.lid[k][1]) return false;
    return a.cam[0] == b.cam[0] && a.cam[1] == b.cam[1] && a.bd == b.bd && a.sf == b.sf && a.sc == b.sc &&
           a.lsf == b.lsf && a.lsc == b.lsc;
}

void set_all_lidars(Candidate& c, int w, int h)
{
    for (int k = 0; k < kLid; ++k) {
        c.lid[k][0] = w;
        c.lid[k][1] = h;
    }
}

int n_lidars(const gsr_plan* p)
{
    int n = 0;
    for (int i = 0; i < p->n_sensors; ++i) n += p->sensors[i].kind == GSR_SENSOR_LIDAR;
    return n;
}

// The plan of a candidate: the input plan's sensors and capacity with every
// camera on cand.cam and the plan's list split, LiDAR k on cand.lid[k] and
// its own split, and cand.bd staged.
gsr_status candidate_plan(const gsr_plan* base, const Candidate& c, gsr_plan* out)
{
    gsr_sensor sensors[GSR_MAX_SENSORS];
    int li = 0;
    for (int i = 0; i < base->n_sensors; ++i) {
        sensors[i] = base->sensors[i];
        const bool lidar = sensors[i].kind == GSR_SENSOR_LIDAR;
        const int* t = lidar ? c.lid[li < kLid ? li : kLid - 1] : c.cam;
        li += lidar;
        sensors[i].tile_w = t[0];
        sensors[i].tile_h = t[1];
        sensors[i].split_first = lidar ? c.lsf : 0;
        sensors[i].split_chunk = lidar ? c.lsc : 0;
    }
    gsr_tiling tiling = base->tiling;
    tiling.batch_depth = c.bd;
    tiling.split_first = c.sf;
    tiling.split_chunk = c.sc;
    return gsr_plan_init(out, base->n_surfels, sensors, base->n_sensors, &tiling, base->max_dup);
}

// List split of the plan's first LiDAR (0 = the plan's).
void plan_lidar_split(const gsr_plan* p, int& sf, int& sc)
{
    sf = sc = 0;
    for (int i = 0; i < p->n_sensors; ++i)
        if (p->sensors[i].kind == GSR_SENSOR_LIDAR) {
            sf = p->sensors[i].split_first;
            sc = p->sensors[i].split_chunk;
            return;
        }
}

// Tile of the plan's first camera of either model (the plan's tiling when
// absent).
void plan_camera_tile(const gsr_plan* p, int t[2])
{
    t[0] = p->tiling.tile_w;
    t[1] = p->tiling.tile_h;
    for (int i = 0; i < p->n_sensors; ++i)
        if (p->sensors[i].kind != GSR_SENSOR_LIDAR) {
            t[0] = p->sensors[i].tile_w;
            t[1] = p->sensors[i].tile_h;
            return;
        }
}

// Tiles of the plan's LiDARs in plan order (the plan's tiling when absent;
// slots past the last LiDAR repeat it).
void plan_lidar_tiles(const gsr_plan* p, int t[kLid][2])
{
    int k = 0;
    int last[2] = {p->tiling.tile_w, p->tiling.tile_h};
    for (int i = 0; i < p->n_sensors && k < kLid; ++i)
        if (p->sensors[i].kind == GSR_SENSOR_LIDAR) {
            last[0] = t[k][0] = p->sensors[i].tile_w;
            last[1] = t[k][1] = p->sensors[i].tile_h;
            ++k;
        }
    for (; k < kLid; ++k) {
        t[k][0] = last[0];
        t[k][1] = last[1];
    }
}

Candidate plan_candidate(const gsr_plan* p)
{
    Candidate c;
    plan_camera_tile(p, c.cam);
    plan_lidar_tiles(p, c.lid);
    c.bd = p->tiling.batch_depth;
    c.sf = p->tiling.split_first;
    c.sc = p->tiling.split_chunk;
    plan_lidar_split(p, c.lsf, c.lsc);
    return c;
}

// Every tile combination the descent can reach (the workspace depends on
// the tiles only): each camera tile with each LiDAR tile for every LiDAR,
// and with every mix of LiDAR tiles over the first two LiDARs.
std::vector<Candidate> all_candidates(const gsr_autotune_space* sp, Candidate start, int nlid)
{
    std::vector<Candidate> v{start};
    const int nc = sp->n_camera_tiles > 0 ? sp->n_camera_tiles : 1;
    const int nl = sp->n_lidar_tiles > 0 ? sp->n_lidar_tiles : 1;
    for (int i = 0; i < nc; ++i)
        for (int j = 0; j < nl; ++j)
            for (int j2 = 0; j2 < (nlid > 1 ? nl : 1); ++j2) {
                Candidate c = start;
                if (sp->n_camera_tiles) {
                    c.cam[0] = sp->camera_tiles[i][0];
                    c.cam[1] = sp->camera_tiles[i][1];
                }
                if (sp->n_lidar_tiles) {
                    set_all_lidars(c, sp->lidar_tiles[j][0], sp->lidar_tiles[j][1]);
                    if (nlid > 1)  // LiDAR 1's tile also stands for the later ones
                        for (int m = 1; m < kLid; ++m) {
                            c.lid[m][0] = sp->lidar_tiles[j2][0];
                            c.lid[m][1] = sp->lidar_tiles[j2][1];
                        }
                }
                v.push_back(c);
            }
    return v;
}

bool space_ok(const gsr_autotune_space* sp)
{
    if (!sp || sp->reps < 1 || sp->warmup < 0) return false;
    if (sp->n_camera_tiles < 0 || sp->n_camera_tiles > GSR_AUTOTUNE_MAX) return false;
    if (sp->n_lidar_tiles < 0 || sp->n_lidar_tiles > GSR_AUTOTUNE_MAX) return false;
    if (sp->n_batch_depths < 0 || sp->n_batch_depths > GSR_AUTOTUNE_MAX) return false;
    if (sp->n_split_firsts < 0 || sp->n_split_firsts > GSR_AUTOTUNE_MAX) return false;
    if (sp->n_split_chunks < 0 || sp->n_split_chunks > GSR_AUTOTUNE_MAX) return false;
    if (sp->n_lidar_split_firsts < 0 || sp->n_lidar_split_firsts > GSR_AUTOTUNE_MAX) return false;
    if (sp->n_lidar_split_chunks < 0 || sp->n_lidar_split_chunks > GSR_AUTOTUNE_MAX) return false;
    return true;
}

}  // namespace

extern "C" gsr_status gsr_autotune_workspace_size(const gsr_plan* plan, const gsr_autotune_space* space,
                                                  size_t* bytes)
{
    if (!plan || !bytes || !space_ok(space)) return GSR_ERR_INVALID_ARG;
    size_t best = 0;
    const int nlid = n_lidars(plan);
    for (const Candidate& c : all_candidates(space, plan_candidate(plan), nlid)) {
        gsr_plan p;
        const gsr_status st = candidate_plan(plan, c, &p);
        if (st != GSR_OK) return st;
        if (p.workspace_bytes > best) best = (size_t)p.workspace_bytes;
    }
    *bytes = best;
    return GSR_OK;
}

extern "C" gsr_status gsr_autotune(const gsr_plan* plan, const gsr_surfels* parts, int32_t n_parts,
                                   const gsr_objects* objects, const gsr_autotune_space* space, void* workspace,
                                   size_t workspace_bytes, const gsr_camera_out* camera_outs,
                                   const gsr_lidar_out* lidar_outs, gsr_autotune_result* result, void* stream)
{
    if (!plan || !parts || n_parts < 1 || !result || !space_ok(space)) return GSR_ERR_INVALID_ARG;
    int64_t total = 0;
    for (int i = 0; i < n_parts; ++i) total += parts[i].n;
    if (total != plan->n_surfels) return GSR_ERR_INVALID_ARG;
    size_t need = 0;
    gsr_status st = gsr_autotune_workspace_size(plan, space, &need);
    if (st != GSR_OK) return st;
    if (!workspace || workspace_bytes < need) return GSR_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::memset(result, 0, sizeof(*result));

    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return gsr::cuda_status(cudaGetLastError());
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return gsr::cuda_status(cudaGetLastError());
    }
    auto frame = [&](const gsr_plan* p) -> gsr_status {
        int first = 0;
        for (int i = 0; i < n_parts; ++i) {
            gsr_status r = gsr_preprocess_part(p, &parts[i], objects, first, workspace, workspace_bytes, stream);
            if (r != GSR_OK) return r;
            first += parts[i].n;
        }
        gsr_status r = gsr_bin_sort(p, workspace, workspace_bytes, stream);
        if (r != GSR_OK) return r;
        return gsr_render_rig(p, workspace, workspace_bytes, camera_outs, lidar_outs, stream);
    };
    // mean frame ms of a candidate, or -1 if its frame failed on the device
    auto measure = [&](const Candidate& c, float& ms) -> gsr_status {
        gsr_plan p;
        gsr_status r = candidate_plan(plan, c, &p);
        if (r != GSR_OK) return r;
        for (int i = 0; i < space->warmup; ++i)
            if ((r = frame(&p)) != GSR_OK) return r;
        if (cudaEventRecord(e0, s) != cudaSuccess) return gsr::cuda_status(cudaGetLastError());
        for (int i = 0; i < space->reps; ++i)
            if ((r = frame(&p)) != GSR_OK) return r;
        if (cudaEventRecord(e1, s) != cudaSuccess) return gsr::cuda_status(cudaGetLastError());
        int32_t dev_status = 0;
        if ((r = gsr_read_status(&p, workspace, &dev_status, nullptr, nullptr, stream)) != GSR_OK) return r;
        float t = 0.f;
        const cudaError_t ce = cudaEventElapsedTime(&t, e0, e1);
        if (ce != cudaSuccess) return gsr::cuda_status(ce);
        ms = dev_status == GSR_OK ? t / space->reps : -1.f;
        return GSR_OK;
    };

    Candidate best = plan_candidate(plan);
    const int nlid = n_lidars(plan);
    float best_ms = -1.f;
    std::vector<std::pair<Candidate, float>> seen;
    auto visit = [&](const Candidate& c) -> gsr_status {
        for (auto& kv : seen)
            if (same(kv.first, c)) return GSR_OK;
        float ms = -1.f;
        gsr_status r = measure(c, ms);
        if (r != GSR_OK) return r;
        seen.push_back({c, ms});
        if (result->n_tried < (int)(sizeof(result->tried) / sizeof(result->tried[0]))) {
            gsr_autotune_trial& t = result->tried[result->n_tried++];
            t.camera_tile[0] = c.cam[0]; t.camera_tile[1] = c.cam[1];
            t.lidar_tile[0] = c.lid[0][0]; t.lidar_tile[1] = c.lid[0][1];
            for (int k = 0; k < kLid; ++k) {
                t.lidar_tiles[k][0] = c.lid[k][0];
                t.lidar_tiles[k][1] = c.lid[k][1];
            }
            t.batch_depth = c.bd;
            t.split_first = c.sf;
            t.split_chunk = c.sc;
            t.lidar_split_first = c.lsf;
            t.lidar_split_chunk = c.lsc;
            t.ms = ms;
        }
        if (ms >= 0.f && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best = c;
        }
        return GSR_OK;
    };
    gsr_status r = visit(best);
    for (int i = 0; r == GSR_OK && i < space->n_camera_tiles; ++i) {
        Candidate c = best;
        c.cam[0] = space->camera_tiles[i][0];
        c.cam[1] = space->camera_tiles[i][1];
        r = visit(c);
    }
    for (int i = 0; r == GSR_OK && i < space->n_lidar_tiles; ++i) {
        Candidate c = best;
        set_all_lidars(c, space->lidar_tiles[i][0], space->lidar_tiles[i][1]);
        r = visit(c);
    }
    // each LiDAR's tile on its own (the workspace bound covers mixes of the
    // first two; later LiDARs keep the common tile)
    for (int k = 0; nlid > 1 && k < 2 && k < nlid; ++k)
        for (int i = 0; r == GSR_OK && i < space->n_lidar_tiles; ++i) {
            Candidate c = best;
            c.lid[k][0] = space->lidar_tiles[i][0];
            c.lid[k][1] = space->lidar_tiles[i][1];
            if (k == 1)  // LiDAR 1's tile also stands for the later ones
                for (int m = 2; m < kLid; ++m) {
                    c.lid[m][0] = c.lid[1][0];
                    c.lid[m][1] = c.lid[1][1];
                }
            r = visit(c);
        }
    for (int i = 0; r == GSR_OK && i < space->n_batch_depths; ++i) {
        Candidate c = best;
        c.bd = space->batch_depths[i];
        r = visit(c);
    }
    for (int i = 0; r == GSR_OK && i < space->n_split_firsts; ++i) {
        Candidate c = best;
        c.sf = space->split_firsts[i];
        r = visit(c);
    }
    for (int i = 0; r == GSR_OK && i < space->n_split_chunks; ++i) {
        Candidate c = best;
        c.sc = space->split_chunks[i];
        r = visit(c);
    }
    for (int i = 0; r == GSR_OK && i < space->n_lidar_split_firsts; ++i) {
        Candidate c = best;
        c.lsf = space->lidar_split_firsts[i];
        r = visit(c);
    }
    for (int i = 0; r == GSR_OK && i < space->n_lidar_split_chunks; ++i) {
        Candidate c = best;
        c.lsc = space->lidar_split_chunks[i];
        r = visit(c);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (r != GSR_OK) return r;
    result->best_ms = best_ms;
    return candidate_plan(plan, best, &result->plan);
}
