// Batched evaluation: many problems per sweep launch, optionally replayed as a CUDA graph.
//
// Problems of one shape (levels, subsystems), solver, kernel family and tile size (threads)
// form a group; a group's sweep launch takes the concatenation of its problems' tile lists (each
// tile names its problem), so problems of different durations and window counts share every
// wave of the GPU instead of each filling a fraction of it, and no tile runs with more threads
// than its own problem's.  The groups' launches of one sweep run concurrently, each on a stream
// of its own forked from the caller's stream and joined back.  The per-problem steps (controls,
// terminal conditions, final reductions) stay per problem.  With MSQOC_BATCH_GRAPH the whole sequence is captured once
// into a CUDA graph and replayed; every buffer it touches belongs to the problems and stays
// where it is, so replays only need the problems' inputs staged with msqoc_set_inputs.
#include <algorithm>
#include <new>
#include <vector>

#include "msqoc_host.h"

using namespace msqoc;

struct msqoc_batch {
    struct Group {
        int L = 0, q = 0, solver = 0, pair = 0, lean = 0;   // shape, solver and kernel family of the group
        int nthreads = 0;                          // threads of its tiles
        std::vector<int> members;     // indices into probs
        SweepArgs args{};             // pds / tiles / lanemap / geometry of the group's launches
        int ntiles = 0;
        int nseg_max = 1;
        ProbDev* pds = nullptr;
        Tile* tiles = nullptr;
        int* lanemap = nullptr;
        std::vector<Tile> host_tiles;         // the group's tiles, longest windows first
        std::vector<int> first, count;        // per member: its tiles in host_tiles (by member k)
        Tile* slot_tiles[MSQOC_BATCH_SLOTS] = {};   // per slot: the tiles of a subset evaluation
        Tile* slot_host[MSQOC_BATCH_SLOTS] = {};    // pinned staging of those tiles
    };
    std::vector<msqoc_problem*> probs;
    std::vector<int> group_of, member_of;   // per problem: its group and index within it
    std::vector<Group> groups;
    int flags = 0;
    int device = 0;
    cudaStream_t cap = nullptr;                   // capture stream (graph mode)
    cudaGraphExec_t exec[2] = {nullptr, nullptr};  // [objective, gradient]
    cudaEvent_t slot_done[MSQOC_BATCH_SLOTS] = {};  // the slot's staging copies have been read
    // per stream set (one per subset slot, the last for whole-batch evaluations): the groups'
    // streams, the fork event on the caller's stream and each group's join event
    std::vector<cudaStream_t> gstream[MSQOC_BATCH_SLOTS + 1];
    std::vector<cudaEvent_t> gjoin[MSQOC_BATCH_SLOTS + 1];
    cudaEvent_t gfork[MSQOC_BATCH_SLOTS + 1] = {};
};

namespace {

void free_batch(msqoc_batch* b) {
    for (auto& g : b->groups) {
        if (g.pds) cudaFree(g.pds);
        if (g.tiles) cudaFree(g.tiles);
        if (g.lanemap) cudaFree(g.lanemap);
        for (int k = 0; k < MSQOC_BATCH_SLOTS; ++k) {
            if (g.slot_tiles[k]) cudaFree(g.slot_tiles[k]);
            if (g.slot_host[k]) cudaFreeHost(g.slot_host[k]);
        }
    }
    for (auto& e : b->slot_done)
        if (e) cudaEventDestroy(e);
    for (int k = 0; k <= MSQOC_BATCH_SLOTS; ++k) {
        for (cudaStream_t gs : b->gstream[k])
            if (gs) cudaStreamDestroy(gs);
        for (cudaEvent_t e : b->gjoin[k])
            if (e) cudaEventDestroy(e);
        if (b->gfork[k]) cudaEventDestroy(b->gfork[k]);
    }
    for (auto& e : b->exec)
        if (e) cudaGraphExecDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
}

// One sweep of every group with tiles, each group's launches issued by launch(gi, stream): on
// the caller's stream s when at most one group has tiles, else concurrently on the groups'
// streams of stream set `set`, forked from s and joined back into it (both also under graph
// capture, where the fork and join become the graph's branches).
template <typename F>
msqoc_status for_groups(msqoc_batch* b, const int* ntiles, int set, cudaStream_t s, F&& launch) {
    const int ng = static_cast<int>(b->groups.size());
    int active = 0;
    for (int gi = 0; gi < ng; ++gi) active += ntiles[gi] > 0;
    if (active <= 1 || b->gstream[set].empty()) {
        for (int gi = 0; gi < ng; ++gi)
            if (ntiles[gi] > 0) CUDA_TRY(launch(gi, s));
        return MSQOC_OK;
    }
    CUDA_TRY(cudaEventRecord(b->gfork[set], s));
    for (int gi = 0; gi < ng; ++gi) {
        if (ntiles[gi] <= 0) continue;
        cudaStream_t gs = b->gstream[set][gi];
        CUDA_TRY(cudaStreamWaitEvent(gs, b->gfork[set], 0));
        CUDA_TRY(launch(gi, gs));
        CUDA_TRY(cudaEventRecord(b->gjoin[set][gi], gs));
        CUDA_TRY(cudaStreamWaitEvent(s, b->gjoin[set][gi], 0));
    }
    return MSQOC_OK;
}

// The launch sequence of one batched evaluation of the problems `sel` (all when sel is empty);
// tiles[g] / ntiles[g] are the tiles of group g to launch; set: the stream set of the groups.
msqoc_status enqueue(msqoc_batch* b, const std::vector<msqoc_problem*>& sel, Tile* const* tiles, const int* ntiles,
                     bool grad, int set, cudaStream_t s) {
    msqoc_status st;
    for (msqoc_problem* p : sel)
        if ((st = launch_controls(p, s))) return st;
    st = for_groups(b, ntiles, set, s, [&](int gi, cudaStream_t gs) {
        SweepArgs a = b->groups[gi].args;
        a.tiles = tiles[gi];
        a.mode = grad ? SWEEP_HISTORY : SWEEP_OBJECTIVE;
        a.seg = 0;
        return launch_sweep(a, ntiles[gi], gs);
    });
    if (st) return st;
    for (msqoc_problem* p : sel)
        if ((st = launch_terminal(p, grad, s))) return st;
    if (!grad) {
        for (msqoc_problem* p : sel) {
            double* o = p->out_dev;
            if ((st = launch_objective_outputs(p, o, o + 1, o + 2, s))) return st;
        }
        return MSQOC_OK;
    }
    st = for_groups(b, ntiles, set, s, [&](int gi, cudaStream_t gs) {
        const auto& g = b->groups[gi];
        for (int seg = g.nseg_max - 1; seg >= 0; --seg) {
            SweepArgs a = g.args;
            a.tiles = tiles[gi];
            a.seg = seg;
            if (g.nseg_max > 1) {
                a.mode = SWEEP_RECOMPUTE;
                const cudaError_t e = launch_sweep(a, ntiles[gi], gs);
                if (e != cudaSuccess) return e;
            }
            a.mode = SWEEP_ADJOINT;
            const cudaError_t e = launch_sweep(a, ntiles[gi], gs);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    });
    if (st) return st;
    for (msqoc_problem* p : sel) {
        const OutLayout ol = out_layout(p->npen, p->pd.d, p->nW);
        double* o = p->out_dev;
        if ((st = launch_gradient_outputs(p, o, o + ol.ga, p->pd.M > 1 ? o + ol.gw : nullptr, s))) return st;
    }
    return MSQOC_OK;
}

msqoc_status enqueue_all(msqoc_batch* b, bool grad, cudaStream_t s) {
    std::vector<Tile*> tiles;
    std::vector<int> ntiles;
    for (auto& g : b->groups) {
        tiles.push_back(g.tiles);
        ntiles.push_back(g.ntiles);
    }
    return enqueue(b, b->probs, tiles.data(), ntiles.data(), grad, MSQOC_BATCH_SLOTS, s);
}

msqoc_status eval(msqoc_batch* b, bool grad, cudaStream_t s) {
    if (grad && !(b->flags & MSQOC_BATCH_GRADIENT))
        return fail(MSQOC_ERR_INVALID_ARG, "batch was created without MSQOC_BATCH_GRADIENT");
    if (!(b->flags & MSQOC_BATCH_GRAPH)) return enqueue_all(b, grad, s);
    cudaGraphExec_t& ex = b->exec[grad ? 1 : 0];
    if (!ex) {
        // capture on a private stream; the first replay below runs it
        CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed));
        const msqoc_status st = enqueue_all(b, grad, b->cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(b->cap, &graph);
        if (st) {
            if (graph) cudaGraphDestroy(graph);
            return st;
        }
        CUDA_TRY(e);
        const cudaError_t ei = cudaGraphInstantiate(&ex, graph, 0);
        cudaGraphDestroy(graph);
        CUDA_TRY(ei);
    }
    CUDA_TRY(cudaGraphLaunch(ex, s));
    return MSQOC_OK;
}

// frees a batch under construction unless released
struct BatchOwner {
    msqoc_batch* b = nullptr;
    ~BatchOwner() {
        if (b) {
            free_batch(b);
            delete b;
        }
    }
};

msqoc_status batch_create(msqoc_problem* const* problems, int32_t n, int32_t flags, msqoc_batch** out) {
    if (!out) return fail(MSQOC_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!problems || n < 1) return fail(MSQOC_ERR_INVALID_ARG, "no problems");
    if (flags & ~(MSQOC_BATCH_GRADIENT | MSQOC_BATCH_GRAPH)) return fail(MSQOC_ERR_INVALID_ARG, "unknown flags %d", flags);
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    for (int i = 0; i < n; ++i) {
        if (!problems[i]) return fail(MSQOC_ERR_INVALID_ARG, "problem %d is NULL", i);
        if (problems[i]->device != dev) return fail(MSQOC_ERR_INVALID_ARG, "problem %d lives on another device", i);
        if (is_shard(problems[i]->pd))
            return fail(MSQOC_ERR_UNSUPPORTED, "problem %d is a window range; batches take whole problems", i);
        for (int j = 0; j < i; ++j)
            if (problems[j] == problems[i]) return fail(MSQOC_ERR_INVALID_ARG, "problem %d appears twice", i);
    }
    BatchOwner owner{new (std::nothrow) msqoc_batch()};
    msqoc_batch* b = owner.b;
    if (!b) return fail(MSQOC_ERR_OUT_OF_MEMORY, "host allocation failed");
    b->flags = flags;
    b->device = dev;
    b->probs.assign(problems, problems + n);
    msqoc_status st = MSQOC_OK;
    // the history buffers first: the problems' device records then hold their final pointers
    if (flags & MSQOC_BATCH_GRADIENT)
        for (msqoc_problem* p : b->probs)
            if (!st) st = ensure_gradient_buffers(p, nullptr);
    if (!st && cudaDeviceSynchronize() != cudaSuccess) st = fail(MSQOC_ERR_CUDA, "synchronize failed");
    // groups by (levels, subsystems, solver, kernel family, tile threads)
    for (int i = 0; i < n && !st; ++i) {
        const ProbDev& pd = b->probs[i]->pd;
        auto it = std::find_if(b->groups.begin(), b->groups.end(), [&](const msqoc_batch::Group& g) {
            return g.L == pd.L && g.q == pd.q && g.solver == pd.solver && g.pair == pd.pair && g.lean == pd.lean &&
                   g.nthreads == pd.nthreads;
        });
        if (it == b->groups.end()) {
            b->groups.emplace_back();
            it = b->groups.end() - 1;
            it->L = pd.L;
            it->q = pd.q;
            it->solver = pd.solver;
            it->pair = pd.pair;
            it->lean = pd.lean;
            it->nthreads = pd.nthreads;
        }
        it->members.push_back(i);
    }
    b->group_of.assign(n, 0);
    b->member_of.assign(n, 0);
    for (size_t gi = 0; gi < b->groups.size(); ++gi)
        for (size_t k = 0; k < b->groups[gi].members.size(); ++k) {
            b->group_of[b->groups[gi].members[k]] = static_cast<int>(gi);
            b->member_of[b->groups[gi].members[k]] = static_cast<int>(k);
        }
    for (auto& g : b->groups) {
        if (st) break;
        int nthreads = 32, cpt = 1, gmax = 1;
        for (int i : g.members) {
            const ProbDev& pd = b->probs[i]->pd;
            nthreads = std::max(nthreads, pd.nthreads);
            cpt = std::max(cpt, pd.cb);
            gmax = std::max(gmax, pd.glocal);
            g.nseg_max = std::max(g.nseg_max, pd.nseg);
        }
        std::vector<ProbDev> pds;
        std::vector<Tile> tiles;
        std::vector<int> maps;
        for (size_t k = 0; k < g.members.size(); ++k) {
            const ProbDev& pd = b->probs[g.members[k]]->pd;
            const int map_base = static_cast<int>(maps.size() / nthreads);
            g.first.push_back(static_cast<int>(tiles.size()));
            g.count.push_back(pd.ntiles);
            for (int t = 0; t < pd.ntiles; ++t) {
                Tile x = tile_at(t, pd.M, pd.E, pd.cb, static_cast<int>(k));
                x.map += map_base;
                tiles.push_back(x);
            }
            const Tile last = tile_at(pd.ntiles - 1, pd.M, pd.E, pd.cb, 0);
            maps.resize(maps.size() + size_t(pd.cb + 1) * nthreads);
            int* mp = maps.data() + size_t(map_base) * nthreads;
            for (int j = 0; j <= pd.cb; ++j)
                build_lanemap(pd.L, pd.q, j < pd.cb ? pd.cb : last.ncol, j < pd.cb ? j + 1 : last.ncol0, nthreads,
                              pd.pair, mp + size_t(j) * nthreads);
            pds.push_back(pd);
        }
        // longest windows first: the CTAs that take longest start in the first wave
        auto tile_len = [&](const Tile& x) {
            const ProbDev& pd = b->probs[g.members[x.prob]]->pd;
            return (pd.nsteps + pd.M - 1) / pd.M;
        };
        g.host_tiles = tiles;
        std::stable_sort(tiles.begin(), tiles.end(), [&](const Tile& x, const Tile& y) { return tile_len(x) > tile_len(y); });
        g.ntiles = static_cast<int>(tiles.size());
        cudaError_t e = cudaMalloc(reinterpret_cast<void**>(&g.pds), pds.size() * sizeof(ProbDev));
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&g.tiles), tiles.size() * sizeof(Tile));
        if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void**>(&g.lanemap), maps.size() * sizeof(int));
        if (e == cudaSuccess) e = cudaMemcpy(g.pds, pds.data(), pds.size() * sizeof(ProbDev), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g.tiles, tiles.data(), tiles.size() * sizeof(Tile), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(g.lanemap, maps.data(), maps.size() * sizeof(int), cudaMemcpyHostToDevice);
        for (int k = 0; k < MSQOC_BATCH_SLOTS && e == cudaSuccess; ++k) {
            e = cudaMalloc(reinterpret_cast<void**>(&g.slot_tiles[k]), tiles.size() * sizeof(Tile));
            if (e == cudaSuccess) e = cudaMallocHost(reinterpret_cast<void**>(&g.slot_host[k]), tiles.size() * sizeof(Tile));
        }
        if (e != cudaSuccess) {
            st = fail(e == cudaErrorMemoryAllocation ? MSQOC_ERR_OUT_OF_MEMORY : MSQOC_ERR_CUDA, "batch tables: %s",
                      cudaGetErrorString(e));
            break;
        }
        const ProbDev& p0 = b->probs[g.members[0]]->pd;
        g.args = sweep_args(p0, g.pds, g.tiles, g.lanemap, SWEEP_OBJECTIVE, 0);
        // one history depth for the launch: the smallest of the members' (it always fits)
        for (int mi : g.members) g.args.hdepth = std::min(g.args.hdepth, b->probs[mi]->pd.hdepth);
        g.args.cpt = cpt;
        g.args.gmax = gmax;
        g.args.nthreads = nthreads;
        SweepArgs adj = g.args;
        adj.mode = SWEEP_ADJOINT;
        if (std::max(sweep_smem_bytes(g.args), sweep_smem_bytes(adj)) > 227 * 1024) {
            st = fail(MSQOC_ERR_UNSUPPORTED, "batched tiles need too much shared memory");
            break;
        }
        // set the kernels' shared-memory limits now (a launch of no tiles only does that), so
        // that a graph capture later makes no attribute calls
        if (launch_sweep(g.args, 0, nullptr) != cudaSuccess || launch_sweep(adj, 0, nullptr) != cudaSuccess)
            st = fail(MSQOC_ERR_CUDA, "sweep kernel attributes could not be set");
    }
    if (!st && (flags & MSQOC_BATCH_GRAPH) && cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess)
        st = fail(MSQOC_ERR_CUDA, "capture stream creation failed");
    for (int k = 0; k < MSQOC_BATCH_SLOTS && !st; ++k)
        if (cudaEventCreateWithFlags(&b->slot_done[k], cudaEventDisableTiming) != cudaSuccess)
            st = fail(MSQOC_ERR_CUDA, "event creation failed");
    // the groups' streams and events (several groups only)
    const size_t ng = b->groups.size();
    for (int k = 0; k <= MSQOC_BATCH_SLOTS && !st && ng > 1; ++k) {
        b->gstream[k].assign(ng, nullptr);
        b->gjoin[k].assign(ng, nullptr);
        cudaError_t e = cudaEventCreateWithFlags(&b->gfork[k], cudaEventDisableTiming);
        for (size_t gi = 0; gi < ng && e == cudaSuccess; ++gi) {
            e = cudaStreamCreateWithFlags(&b->gstream[k][gi], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->gjoin[k][gi], cudaEventDisableTiming);
        }
        if (e != cudaSuccess) st = fail(MSQOC_ERR_CUDA, "group streams: %s", cudaGetErrorString(e));
    }
    if (st) return st;
    *out = b;
    owner.b = nullptr;
    return MSQOC_OK;
}

msqoc_status batch_eval_subset(msqoc_batch* b, const int32_t* members, int32_t n, int32_t gradient, int32_t slot,
                               void* stream) {
    if (!b || !members || n < 1) return fail(MSQOC_ERR_INVALID_ARG, "batch or members is NULL / empty");
    if (slot < 0 || slot >= MSQOC_BATCH_SLOTS) return fail(MSQOC_ERR_INVALID_ARG, "slot %d out of range", slot);
    if (gradient && !(b->flags & MSQOC_BATCH_GRADIENT))
        return fail(MSQOC_ERR_INVALID_ARG, "batch was created without MSQOC_BATCH_GRADIENT");
    const int np = static_cast<int>(b->probs.size());
    std::vector<char> seen(np, 0);
    for (int i = 0; i < n; ++i) {
        if (members[i] < 0 || members[i] >= np) return fail(MSQOC_ERR_INVALID_ARG, "member %d out of range", members[i]);
        if (seen[members[i]]++) return fail(MSQOC_ERR_INVALID_ARG, "member %d listed twice", members[i]);
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the slot's staging buffers are rewritten only after its previous copies were read
    CUDA_TRY(cudaEventSynchronize(b->slot_done[slot]));
    std::vector<msqoc_problem*> sel;
    std::vector<Tile*> tiles(b->groups.size());
    std::vector<int> ntiles(b->groups.size(), 0);
    for (int i = 0; i < n; ++i) sel.push_back(b->probs[members[i]]);
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        auto& g = b->groups[gi];
        Tile* h = g.slot_host[slot];
        int cnt = 0;
        for (int i = 0; i < n; ++i) {
            if (b->group_of[members[i]] != static_cast<int>(gi)) continue;
            const int k = b->member_of[members[i]];
            std::copy(g.host_tiles.begin() + g.first[k], g.host_tiles.begin() + g.first[k] + g.count[k], h + cnt);
            cnt += g.count[k];
        }
        auto tile_len = [&](const Tile& x) {
            const ProbDev& pd = b->probs[g.members[x.prob]]->pd;
            return (pd.nsteps + pd.M - 1) / pd.M;
        };
        std::stable_sort(h, h + cnt, [&](const Tile& x, const Tile& y) { return tile_len(x) > tile_len(y); });
        if (cnt) CUDA_TRY(cudaMemcpyAsync(g.slot_tiles[slot], h, cnt * sizeof(Tile), cudaMemcpyHostToDevice, s));
        tiles[gi] = g.slot_tiles[slot];
        ntiles[gi] = cnt;
    }
    CUDA_TRY(cudaEventRecord(b->slot_done[slot], s));
    return enqueue(b, sel, tiles.data(), ntiles.data(), gradient != 0, slot, s);
}

}  // namespace

extern "C" {

msqoc_status msqoc_batch_create(msqoc_problem* const* problems, int32_t n, int32_t flags, msqoc_batch** out) {
    if (out) *out = nullptr;
    return guarded([&] { return batch_create(problems, n, flags, out); });
}

msqoc_status msqoc_batch_eval_objective(msqoc_batch* b, void* stream) {
    if (!b) return fail(MSQOC_ERR_INVALID_ARG, "batch is NULL");
    return guarded([&] { return eval(b, false, static_cast<cudaStream_t>(stream)); });
}

msqoc_status msqoc_batch_eval_gradient(msqoc_batch* b, void* stream) {
    if (!b) return fail(MSQOC_ERR_INVALID_ARG, "batch is NULL");
    return guarded([&] { return eval(b, true, static_cast<cudaStream_t>(stream)); });
}

msqoc_status msqoc_batch_eval_subset(msqoc_batch* b, const int32_t* members, int32_t n, int32_t gradient,
                                     int32_t slot, void* stream) {
    return guarded([&] { return batch_eval_subset(b, members, n, gradient, slot, stream); });
}

msqoc_status msqoc_batch_destroy(msqoc_batch* b) {
    if (!b) return MSQOC_OK;
    cudaDeviceSynchronize();
    free_batch(b);
    delete b;
    return MSQOC_OK;
}

msqoc_status msqoc_set_inputs(msqoc_problem* p, const double* alpha, const double* W, void* stream) {
    if (!p) return fail(MSQOC_ERR_INVALID_ARG, "problem is NULL");
    return stage_inputs(p, alpha, W, static_cast<cudaStream_t>(stream));
}

msqoc_status msqoc_get_objective(msqoc_problem* p, double* P_out, double* J_out, double* pen_out, void* stream) {
    if (!p || !P_out) return fail(MSQOC_ERR_INVALID_ARG, "problem or P_out is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double* o = p->out_dev;
    CUDA_TRY(cudaMemcpyAsync(P_out, o, sizeof(double), cudaMemcpyDefault, s));
    if (J_out) CUDA_TRY(cudaMemcpyAsync(J_out, o + 1, sizeof(double), cudaMemcpyDefault, s));
    if (pen_out && p->pd.M > 1)
        CUDA_TRY(cudaMemcpyAsync(pen_out, o + 2, (p->pd.M - 1) * sizeof(double), cudaMemcpyDefault, s));
    const bool host = !is_device_ptr(P_out) || (J_out && !is_device_ptr(J_out)) || (pen_out && !is_device_ptr(pen_out));
    return host ? check_status_sync(p, s) : MSQOC_OK;
}

msqoc_status msqoc_get_gradient(msqoc_problem* p, double* P_out, double* grad_alpha, double* grad_W, void* stream) {
    if (!p || !grad_alpha) return fail(MSQOC_ERR_INVALID_ARG, "problem or grad_alpha is NULL");
    if (p->pd.M > 1 && !grad_W) return fail(MSQOC_ERR_INVALID_ARG, "grad_W is NULL but M > 1");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double* o = p->out_dev;
    const OutLayout ol = out_layout(p->npen, p->pd.d, p->nW);
    if (P_out) CUDA_TRY(cudaMemcpyAsync(P_out, o, sizeof(double), cudaMemcpyDefault, s));
    CUDA_TRY(cudaMemcpyAsync(grad_alpha, o + ol.ga, p->pd.d * sizeof(double), cudaMemcpyDefault, s));
    if (p->pd.M > 1) CUDA_TRY(cudaMemcpyAsync(grad_W, o + ol.gw, p->nW * sizeof(double), cudaMemcpyDefault, s));
    const bool host = (P_out && !is_device_ptr(P_out)) || !is_device_ptr(grad_alpha) ||
                      (p->pd.M > 1 && !is_device_ptr(grad_W));
    return host ? check_status_sync(p, s) : MSQOC_OK;
}

}  // extern "C"
