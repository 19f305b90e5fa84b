// C-ABI of the library: context, molecule/basis/grid loading, integration driver.
//
// The driver follows Algorithm 2 on one device: the plan is built once per
// geometry and stays resident (grid points, partition weights, batch lists);
// each integration copies P in (unless it already lives on the device), walks
// the batches in chunks that fit the scratch budget (the paper's
// memory-saturating device subsets), and reduces E, N and V on the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <deque>
#include <mutex>
#include <thread>
#include <tuple>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <vector>

#include "internal.h"
#include "mixed.h"

using namespace gbxc;

namespace {

struct Schedule {
    int precision = -1;
    int b0 = -1, b1 = -1;
    size_t budget = 0;
    struct Chunk {
        int64_t t0, t1, row0, rows;
        int max_nfunc;
        int64_t task0, ntask;
    };
    std::vector<Chunk> chunks;
    int *d_tasks = nullptr;     // 5 ints per task
    int64_t ntasks = 0;
    int64_t max_rows = 0;
    MixedSchedule mixed;        // extra state of the mixed form
};
using SchedKey = std::tuple<int, int, int, size_t, int>;   // precision, b0, b1, scratch budget, N tile

struct Molecule {
    int natoms = 0, nshell = 0, nbf = 0;
    std::vector<double> xyz;
    std::vector<int> Z;
    std::vector<DevShell> shells;
    DevShell *d_shells = nullptr;
    double *d_atoms = nullptr, *d_rnn = nullptr;
    int *d_nbr = nullptr;           // natoms x (natoms - 1) neighbours of each atom by distance
    double *d_nbr_r = nullptr;      // and their distances
    bool has_grid = false;
    gbxc_grid_spec spec{};
    HostPlan plan;
    DevPlan dev;
    std::vector<void *> dev_allocs;
    double *d_tileE = nullptr, *d_tileN = nullptr, *d_Eb = nullptr, *d_Nb = nullptr;
    int64_t *d_point_index = nullptr;   // device-planned molecules: generation index of each point
    std::map<SchedKey, std::unique_ptr<Schedule>> scheds;
    MixedResident mixed_res;
    double work = 0.0;          // sum_j W_j, for balancing many molecules over graph branches
    double *many_P = nullptr, *many_V = nullptr, *many_tot = nullptr;   // gbxc_integrate_many
    double *many_Vacc = nullptr;    // its V accumulator in the grouped launch
    float *many_pdf = nullptr;      // and its P region (double-float pairs, slices; tensor-core form)
    size_t many_cap = 0;
};

// Everything one in-flight integration owns on the device.  A workspace either owns its
// buffers (cudaMalloc, grown on demand) or has them carved from the context's arena.
struct Workspace {
    cudaStream_t stream = nullptr;
    bool owns = true;
    void *scratch = nullptr;
    size_t scratch_cap = 0;
    double *d_P = nullptr, *d_Vacc = nullptr, *d_V = nullptr, *d_tot = nullptr;
    size_t mat_cap = 0;
    double *tileE = nullptr, *tileN = nullptr, *Eb = nullptr, *Nb = nullptr;
    size_t tile_cap = 0, batch_cap = 0;
    MixedCtx mixed;
    double *d_P2 = nullptr, *d_Vacc2 = nullptr, *d_V2 = nullptr;   // second spin (unrestricted)
    size_t mat2_cap = 0;
};

// First-fit allocator over one device allocation (the paper's preallocated device arena
// managed by hand, Sec. 2.3).
struct Arena {
    char *base = nullptr;
    size_t cap = 0;
    std::map<size_t, size_t> free_;   // offset -> bytes
    void init(char *b, size_t c) {
        base = b;
        cap = c;
        free_.clear();
        if (c) free_[0] = c;
    }
    static size_t up(size_t b) { return (b + 255) & ~(size_t)255; }
    bool alloc(size_t bytes, size_t *off) {
        bytes = up(std::max<size_t>(bytes, 256));
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            size_t rest = it->second - bytes, o = it->first;
            free_.erase(it);
            if (rest) free_[o + bytes] = rest;
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = up(std::max<size_t>(bytes, 256));
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t free_bytes() const {
        size_t f = 0;
        for (auto &kv : free_) f += kv.second;
        return f;
    }
};

// One queued or running request of the serving loop.
struct Request {
    long long ticket = 0;
    int mol = 0, functional = 0, precision = 0;
    std::vector<double> P, V;
    double E = 0.0, N = 0.0;
    int state = 0;              // 0 queued, 1 running, 2 done
    int status = GBXC_OK;
    std::string err;
    size_t off = 0, bytes = 0;
    int slot = -1;
    double *pin_tot = nullptr;
    std::chrono::steady_clock::time_point t_submit, t_done;
};

struct Server {
    bool running = false;
    int nslots = 0;
    size_t slot_budget = 0;     // scratch budget of one request's schedule
    char *arena_mem = nullptr;
    Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done_ev;
    std::vector<double *> pin;  // per slot: pinned P/V staging (2 nbf^2) + totals
    std::vector<size_t> pin_cap;
    std::vector<std::shared_ptr<Request>> slot_req;
    std::vector<Workspace> slot_ws;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<long long, std::shared_ptr<Request>> tickets;
    long long next_ticket = 1;
    std::mutex qmu;             // queue, tickets and request states
    std::condition_variable cv; // request completion and new submissions
    std::atomic<bool> stop{false};
    std::thread thread;
    long long admitted = 0, completed = 0;
};

// A captured CUDA graph of gbxc_integrate_many for one molecule list.
struct ManyGraph {
    std::vector<int> mols, fns;
    int precision = -1, branches = 0, tile_n = 0;
    size_t budget = 0;
    cudaGraphExec_t exec = nullptr;
    long long launches[GBXC_NKERNEL] = {};
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
};

// gbxc_integrate_many as one grouped launch per kernel and chunk: the molecules' plans are
// concatenated into one combined plan (points copied; batches, shells and tiles renumbered;
// function indices kept local to each molecule, since P and V are per molecule), so each
// kernel launch of a chunk spans the tiles of every molecule in it.  batch_mol and the MolRef
// table give each batch its molecule's P, V accumulator, nbf and functional.  The launches of
// one call are captured once into a CUDA graph.
struct Group {
    std::vector<int> mols;
    int precision = -1, tile_n = 0;
    size_t budget = 0;
    Molecule gm;                       // the combined plan; owns its device copies
    std::vector<int> bofs;             // first combined batch of each molecule, then the total
    int *d_batch_mol = nullptr;
    MolRef *d_mols = nullptr;
    std::vector<MolRef> h_mols;
    Workspace ws;
    cudaGraphExec_t exec = nullptr;
    long long launches[GBXC_NKERNEL] = {};
};

}  // namespace

struct gbxc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t scratch_budget = 0;
    bool budget_given = false;      // gbxc_create's scratch_bytes (used as is everywhere)
    size_t many_budget = 0;         // the many-molecule calls' budget, fixed at their first call
    Workspace ws;                   // the default workspace (synchronous calls)
    std::vector<Workspace> branch_ws;   // gbxc_integrate_many branches
    ManyGraph many;
    std::unique_ptr<Group> group;   // gbxc_integrate_many, grouped schedule
    // gbxc_autotune results: (molecule list, precision) -> {graph branches, GEMM N tile}
    std::map<std::pair<std::vector<int>, int>, std::pair<int, int>> tuned;
    std::string err;
    std::map<int, std::unique_ptr<Molecule>> mols;
    int next_id = 0;
    Profiler prof;
    std::recursive_mutex mu;        // serialises host-side work on the context
    Server srv;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;   // timing of graph launches (gbxc_autotune)
};

namespace {

struct CudaFail {
    std::string msg;
};

void check(cudaError_t e, const char *what) {
    if (e != cudaSuccess) throw CudaFail{std::string(what) + ": " + cudaGetErrorString(e)};
}

int fail(gbxc_ctx *ctx, int code, const std::string &msg) {
    if (ctx) ctx->err = msg;
    return code;
}

struct ArgError {
    std::string msg;
};

#define REQUIRE(cond, msg)                      \
    do {                                        \
        if (!(cond)) throw ArgError{msg};       \
    } while (0)

template <typename F>
int guarded(gbxc_ctx *ctx, F &&body) {
    std::unique_lock<std::recursive_mutex> lk;
    if (ctx) lk = std::unique_lock<std::recursive_mutex>(ctx->mu);
    try {
        if (ctx) {
            ctx->err.clear();
            if (ctx->device < 0) return body();
            cudaError_t e = cudaSetDevice(ctx->device);
            if (e != cudaSuccess) return fail(ctx, GBXC_ECUDA, cudaGetErrorString(e));
        }
        return body();
    } catch (const ArgError &e) {
        return fail(ctx, GBXC_EINVAL, e.msg);
    } catch (const CudaFail &e) {
        return fail(ctx, GBXC_ECUDA, e.msg);
    } catch (const std::bad_alloc &) {
        return fail(ctx, GBXC_ENOMEM, "host allocation failed");
    } catch (const std::exception &e) {
        return fail(ctx, GBXC_EINVAL, e.what());
    }
}

template <typename T>
T *dev_upload(Molecule &m, const std::vector<T> &v, cudaStream_t s) {
    T *p = nullptr;
    size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
    check(cudaMalloc(&p, bytes), "cudaMalloc plan");
    m.dev_allocs.push_back(p);
    if (!v.empty()) check(cudaMemcpyAsync(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s),
                          "upload plan");
    return p;
}

template <typename T>
T *dev_alloc(Molecule &m, size_t n) {
    T *p = nullptr;
    check(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T)), "cudaMalloc");
    m.dev_allocs.push_back(p);
    return p;
}

void free_schedule(Schedule &s) {
    if (s.d_tasks) cudaFree(s.d_tasks);
    s.d_tasks = nullptr;
    free_mixed_schedule(s.mixed);
    s = Schedule{};
}

void free_schedules(Molecule &m) {
    for (auto &kv : m.scheds) free_schedule(*kv.second);
    m.scheds.clear();
}

void free_grid(Molecule &m) {
    for (void *p : m.dev_allocs) cudaFree(p);
    m.dev_allocs.clear();
    free_schedules(m);
    m.dev = DevPlan{};
    m.has_grid = false;
}

// Every device allocation a loaded molecule holds (basis, grid, plan, schedules, buffers).
void free_molecule(Molecule &m) {
    free_grid(m);
    cudaFree(m.d_shells);
    free_mixed_resident(m.mixed_res);
    cudaFree(m.d_atoms);
    cudaFree(m.d_rnn);
    cudaFree(m.d_nbr);
    cudaFree(m.d_nbr_r);
    cudaFree(m.many_P);
    cudaFree(m.many_V);
    cudaFree(m.many_tot);
    cudaFree(m.many_Vacc);
    cudaFree(m.many_pdf);
}


void free_workspace(Workspace &w) {
    if (w.owns) {
        cudaFree(w.scratch);
        cudaFree(w.d_P);
        cudaFree(w.d_Vacc);
        cudaFree(w.d_V);
        cudaFree(w.d_tot);
        cudaFree(w.tileE);
        cudaFree(w.tileN);
        cudaFree(w.Eb);
        cudaFree(w.Nb);
        cudaFree(w.d_P2);
        cudaFree(w.d_Vacc2);
        cudaFree(w.d_V2);
        free_mixed_ctx(w.mixed);
    }
    w = Workspace{};
}

void free_group(std::unique_ptr<Group> &G);
// The cached grouped launch holds copies of its molecules' plans and their buffers: drop it
// when one of them is unloaded or gets a new grid.
void drop_group_with(gbxc_ctx *ctx, int mol);

void free_group(std::unique_ptr<Group> &G) {
    if (!G) return;
    if (G->exec) cudaGraphExecDestroy(G->exec);
    cudaFree(G->d_batch_mol);
    cudaFree(G->d_mols);
    free_workspace(G->ws);
    free_molecule(G->gm);
    G.reset();
}

void drop_group_with(gbxc_ctx *ctx, int mol) {
    if (ctx->group && std::find(ctx->group->mols.begin(), ctx->group->mols.end(), mol) != ctx->group->mols.end())
        free_group(ctx->group);
}

// The LDA / GGA codes every integration call takes (the meta-GGA has its own paths).
bool semilocal_lda_gga(int functional) {
    return functional == GBXC_SLATER || functional == GBXC_PBE || functional == GBXC_PBE0_SL;
}

bool is_device_ptr(const void *p) {
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

// Device memory that lives on another GPU than `device` (managed memory is reachable from
// every device and does not count).  Kernels of a context run on its own device only, so
// such a buffer is refused instead of being read over the interconnect or faulting.
bool on_other_device(const void *p, int device) {
    cudaPointerAttributes attr;
    cudaError_t e = cudaPointerGetAttributes(&attr, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return attr.type == cudaMemoryTypeDevice && attr.device != device;
}

Molecule &get_mol(gbxc_ctx *ctx, int mol) {
    auto it = ctx->mols.find(mol);
    if (it == ctx->mols.end()) throw ArgError{"unknown molecule id " + std::to_string(mol)};
    return *it->second;
}

template <typename T>
void grow_buf(T *&p, size_t &cap, size_t need, const char *what) {
    if (need <= cap && p) return;
    cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, std::max<size_t>(need, 1) * sizeof(T));
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw CudaFail{std::string(what) + ": allocation of " + std::to_string(need * sizeof(T)) +
                       " bytes failed"};
    }
    cap = need;
}

size_t row_bytes(int precision) { return precision == GBXC_FP64 ? fp64_row_bytes() : mixed_row_bytes(); }

// Device bytes one integration of `m` with schedule `S` needs in a workspace.
size_t footprint(const Molecule &m, const Schedule &S, int precision) {
    size_t nn = (size_t)m.nbf * m.nbf;
    size_t b = (size_t)S.max_rows * row_bytes(precision) + 256;
    b += Arena::up(nn * 8) * 3 + 256;                      // P, V_acc, V (+ totals)
    b += Arena::up((size_t)m.plan.ntiles() * 8) * 2;       // tile E/N partials
    b += Arena::up((size_t)std::max(m.plan.nbatch(), 1) * 8) * 2;
    if (precision == GBXC_MIXED) b += mixed_reserve_bytes(S.mixed, m.nbf) + 4 * 256;
    return b;
}

// Make `w` (an owning workspace) large enough for one integration of `m` with `S`.
void reserve(Workspace &w, const Molecule &m, const Schedule &S, int precision) {
    size_t nn = (size_t)m.nbf * m.nbf;
    if (nn > w.mat_cap || !w.d_P) {
        size_t c0 = w.mat_cap, c1 = w.mat_cap, c2 = w.mat_cap;
        grow_buf(w.d_P, c0, nn, "P");
        grow_buf(w.d_Vacc, c1, nn, "V_acc");
        grow_buf(w.d_V, c2, nn, "V");
        w.mat_cap = nn;
    }
    size_t one = 2;
    if (!w.d_tot) grow_buf(w.d_tot, one, 3, "totals");   // E, N and the non-finite-P flag
    size_t nt = (size_t)m.plan.ntiles(), nb = (size_t)std::max(m.plan.nbatch(), 1);
    if (nt > w.tile_cap || !w.tileE) {
        size_t c0 = w.tile_cap, c1 = w.tile_cap;
        grow_buf(w.tileE, c0, nt, "tile E");
        grow_buf(w.tileN, c1, nt, "tile N");
        w.tile_cap = nt;
    }
    if (nb > w.batch_cap || !w.Eb) {
        size_t c0 = w.batch_cap, c1 = w.batch_cap;
        grow_buf(w.Eb, c0, nb, "batch E");
        grow_buf(w.Nb, c1, nb, "batch N");
        w.batch_cap = nb;
    }
    size_t sb = (size_t)S.max_rows * row_bytes(precision);
    if (sb > w.scratch_cap || !w.scratch) {
        char *p = static_cast<char *>(w.scratch);
        size_t cap = w.scratch_cap;
        grow_buf(p, cap, std::max<size_t>(sb, 256), "scratch");
        w.scratch = p;
        w.scratch_cap = cap;
    }
    if (precision == GBXC_MIXED) check(mixed_reserve(w.mixed, S.mixed, m.nbf), "mixed buffers");
}

// Carve a non-owning workspace for one integration out of `base` (footprint bytes).
void carve(Workspace &w, char *base, const Molecule &m, const Schedule &S, int precision, void *encode_fn) {
    size_t nn = (size_t)m.nbf * m.nbf;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        char *p = base + o;
        o += Arena::up(std::max<size_t>(bytes, 8));
        return p;
    };
    w.owns = false;
    w.scratch = take((size_t)S.max_rows * row_bytes(precision));
    w.scratch_cap = (size_t)S.max_rows * row_bytes(precision);
    w.d_P = reinterpret_cast<double *>(take(nn * 8));
    w.d_Vacc = reinterpret_cast<double *>(take(nn * 8));
    w.d_V = reinterpret_cast<double *>(take(nn * 8));
    w.d_tot = reinterpret_cast<double *>(take(24));   // E, N and the non-finite-P flag
    w.mat_cap = nn;
    w.tileE = reinterpret_cast<double *>(take((size_t)m.plan.ntiles() * 8));
    w.tileN = reinterpret_cast<double *>(take((size_t)m.plan.ntiles() * 8));
    w.tile_cap = (size_t)m.plan.ntiles();
    size_t nb = (size_t)std::max(m.plan.nbatch(), 1);
    w.Eb = reinterpret_cast<double *>(take(nb * 8));
    w.Nb = reinterpret_cast<double *>(take(nb * 8));
    w.batch_cap = nb;
    if (precision == GBXC_MIXED) {
        const MixedSchedule &ms = S.mixed;
        w.mixed = MixedCtx{};
        w.mixed.encode_fn = encode_fn;
        check(mixed_init(w.mixed), "mixed init");
        w.mixed.pslices = reinterpret_cast<uint16_t *>(take((size_t)std::max<int64_t>(ms.max_prows, 1) * 32 * 5 * 2));
        w.mixed.pslice_rows = (size_t)std::max<int64_t>(ms.max_prows, 1) * 32 * 5;
        w.mixed.pdf = reinterpret_cast<float *>(take(mixed_pdf_floats(m.nbf) * 4));
        w.mixed.pdf_cap = mixed_pdf_floats(m.nbf);
        w.mixed.d_err = reinterpret_cast<int *>(take(16));   // error word and GEMM task counter
    }
}

// The default budget is fixed at the first integration of the context (half the free device
// memory then, at most 128 GiB), so schedules stay valid across calls.  Fewer, larger chunks
// pay the ramp-up and tail of each kernel fewer times: the 64-water call runs in 2 chunks
// instead of 5 at 48 GiB.
size_t scratch_budget(gbxc_ctx *ctx) {
    if (ctx->scratch_budget) return ctx->scratch_budget;
    size_t fr = 0, tot = 0;
    check(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
    size_t b = (size_t)(0.5 * (double)fr);
    ctx->scratch_budget = std::min<size_t>(b, (size_t)128 << 30);
    return ctx->scratch_budget;
}

// Memory beside the single-call workspace (the many-molecule branches, the serving arena): a
// default budget is capped by half the device memory free when it is first needed, less the
// part of the single-call budget that its workspace has not allocated yet, so that either
// order of calls fits.
size_t side_budget(gbxc_ctx *ctx, size_t &fixed) {
    if (ctx->budget_given) return scratch_budget(ctx);
    if (fixed) return fixed;
    const size_t b = scratch_budget(ctx);
    size_t fr = 0, tot = 0;
    check(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
    const size_t pending = b > ctx->ws.scratch_cap ? b - ctx->ws.scratch_cap : 0;
    const size_t room = fr > pending ? fr - pending : 0;
    fixed = std::max<size_t>(std::min<size_t>(b, (size_t)(0.5 * (double)room)), (size_t)64 << 20);
    return fixed;
}

// Chunks of tiles whose slabs fit the budget, and the V-contraction tasks of each chunk.
Schedule &get_schedule(Molecule &m, int precision, int b0, int b1, size_t budget, int tile_n = 128) {
    if (precision == GBXC_FP64) tile_n = 128;   // the float64 kernels have one tile shape
    SchedKey key{precision, b0, b1, budget, tile_n};
    auto it = m.scheds.find(key);
    if (it != m.scheds.end()) return *it->second;
    auto sp = std::make_unique<Schedule>();
    Schedule &S = *sp;
    const HostPlan &P = m.plan;
    int64_t max_rows = (int64_t)(budget / row_bytes(precision));
    int64_t tb = P.batch_tile[b0], te = P.batch_tile[b1];
    std::vector<int> tasks;
    int64_t t = tb;
    while (t < te) {
        Schedule::Chunk c;
        c.t0 = t;
        c.row0 = P.tile_row[t];
        while (t < te && P.tile_row[t + 1] - c.row0 <= max_rows) ++t;
        if (t == c.t0) throw CudaFail{"scratch budget too small for one tile"};
        c.t1 = t;
        c.rows = P.tile_row[t] - c.row0;
        c.max_nfunc = 0;
        c.task0 = (int64_t)tasks.size() / 5;
        int j0 = P.tile_batch[c.t0], j1 = P.tile_batch[c.t1 - 1];
        for (int j = j0; j <= j1; ++j) {
            int n = (int)(P.func_ptr[j + 1] - P.func_ptr[j]);
            c.max_nfunc = std::max(c.max_nfunc, n);
            int64_t s0 = std::max(P.batch_tile[j], c.t0), s1 = std::min(P.batch_tile[j + 1], c.t1);
            if (precision == GBXC_FP64)
                append_fp64_vtasks(j, n, s0, s1, tasks);
            else
                append_mixed_vtasks(j, n, s0, s1, tile_n, tasks);
        }
        c.ntask = (int64_t)tasks.size() / 5 - c.task0;
        S.chunks.push_back(c);
        S.max_rows = std::max(S.max_rows, c.rows);
    }
    S.ntasks = (int64_t)tasks.size() / 5;
    if (precision == GBXC_MIXED) {
        std::vector<int64_t> c0, c1;
        for (const auto &c : S.chunks) {
            c0.push_back(c.t0);
            c1.push_back(c.t1);
        }
        build_mixed_schedule(m.plan, c0, c1, tile_n, S.mixed);
    }
    if (!tasks.empty()) {
        check(cudaMalloc(&S.d_tasks, tasks.size() * sizeof(int)), "cudaMalloc tasks");
        check(cudaMemcpy(S.d_tasks, tasks.data(), tasks.size() * sizeof(int), cudaMemcpyHostToDevice),
              "upload tasks");
    }
    S.precision = precision;
    S.b0 = b0;
    S.b1 = b1;
    S.budget = budget;
    Schedule &ref = *sp;
    m.scheds.emplace(key, std::move(sp));
    return ref;
}

// Queue one integration of `m` on stream `s` with workspace `w` (no host synchronisation):
// V_acc <- 0, chunks, V = V_acc + V_acc^T into dV (if non-null), per-batch sums into w.Eb/Nb
// and {E, N} into w.d_tot.
void enqueue(Workspace &w, Molecule &m, const Schedule &S, const double *dP, int functional, int precision,
             int b0, int b1, double *dV, bool batch_sums, cudaStream_t s, Profiler *prof,
             double *d_tot = nullptr) {
    size_t nn = (size_t)m.nbf * m.nbf;
    check(cudaMemsetAsync(w.d_Vacc, 0, nn * 8, s), "zero V");
    if (precision == GBXC_MIXED) check(mixed_begin(w.mixed, dP, m.nbf, s), "mixed begin");
    for (size_t ci = 0; ci < S.chunks.size(); ++ci) {
        const auto &c = S.chunks[ci];
        ChunkArgs a;
        a.plan = m.dev;
        a.shells = m.d_shells;
        a.nbf = m.nbf;
        a.t0 = c.t0;
        a.t1 = c.t1;
        a.row0 = c.row0;
        a.rows = c.rows;
        a.max_nfunc = c.max_nfunc;
        a.functional = functional;
        a.P = dP;
        a.Vacc = w.d_Vacc;
        a.tileE = w.tileE;
        a.tileN = w.tileN;
        a.scratch = w.scratch;
        a.vtasks = S.d_tasks ? S.d_tasks + 5 * c.task0 : nullptr;
        a.nvtasks = (int)c.ntask;
        a.prof = prof;
        if (precision == GBXC_FP64 && functional == GBXC_MVS_X)
            check(launch_fp64_chunk_mgga(a, s), "fp64 meta-GGA chunk");
        else if (precision == GBXC_FP64)
            check(launch_fp64_chunk(a, s), "fp64 chunk");
        else if (functional == GBXC_MVS_X)
            check(launch_mixed_chunk_mgga(a, w.mixed, m.mixed_res, S.mixed, (int)ci, s), "mixed meta-GGA chunk");
        else
            check(launch_mixed_chunk(a, w.mixed, m.mixed_res, S.mixed, (int)ci, s), "mixed chunk");
    }
    if (batch_sums) {
        int nb = std::max(m.plan.nbatch(), 1);
        check(cudaMemsetAsync(w.Eb, 0, nb * 8, s), "zero Eb");
        check(cudaMemsetAsync(w.Nb, 0, nb * 8, s), "zero Nb");
    }
    FinishArgs f;
    f.Vacc = w.d_Vacc;
    f.V = dV;
    f.nbf = m.nbf;
    f.tileE = w.tileE;
    f.tileN = w.tileN;
    f.batch_tile = m.dev.batch_tile;
    f.b0 = b0;
    f.b1 = b1;
    f.Eb = w.Eb;
    f.Nb = w.Nb;
    f.tot = d_tot ? d_tot : w.d_tot;
    f.prof = prof;
    check(launch_finish(f, s), "finish");
}

int integrate_impl(gbxc_ctx *ctx, int mol, const double *P, int functional, int precision, int b0,
                   int b1, double *Exc, double *Vxc, double *Nel, double *Eb, double *Nb,
                   void *stream) {
    REQUIRE(ctx->device >= 0, "integration needs a device context");
    Molecule &m = get_mol(ctx, mol);
    if (!m.has_grid) throw ArgError{"molecule has no grid (call gbxc_load_grid first)"};
    REQUIRE(P, "P is NULL");
    REQUIRE(!on_other_device(P, ctx->device) && (!Vxc || !on_other_device(Vxc, ctx->device)),
            "P or Vxc is memory of another device");
    REQUIRE(semilocal_lda_gga(functional) || functional == GBXC_MVS_X, "unknown functional");
    REQUIRE(precision == GBXC_FP64 || precision == GBXC_MIXED, "unknown precision");
    int nb = m.plan.nbatch();
    REQUIRE(0 <= b0 && b0 <= b1 && b1 <= nb, "batch range out of bounds");
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    size_t nn = (size_t)m.nbf * m.nbf;
    Workspace &w = ctx->ws;
    const Schedule &S = get_schedule(m, precision, b0, b1, scratch_budget(ctx));
    reserve(w, m, S, precision);
    if (precision == GBXC_MIXED && functional == GBXC_MVS_X)
        check(mixed_reserve_mgga(w.mixed, S.max_rows), "mixed meta-GGA buffers");
    const double *dP = P;
    if (!is_device_ptr(P)) {
        check(cudaMemcpyAsync(w.d_P, P, nn * 8, cudaMemcpyHostToDevice, s), "copy P");
        dP = w.d_P;
    }
    double *dV = (Vxc && is_device_ptr(Vxc)) ? Vxc : w.d_V;
    ctx->prof.begin(GBXC_K_FINISH, s);
    check(launch_check_finite(dP, (int64_t)nn, w.d_tot + 2, true, s), "check P");
    ctx->prof.end(GBXC_K_FINISH, s);
    enqueue(w, m, S, dP, functional, precision, b0, b1, Vxc ? dV : nullptr, Eb || Nb, s, &ctx->prof);
    double tot[3];
    check(cudaMemcpyAsync(tot, w.d_tot, 24, cudaMemcpyDeviceToHost, s), "copy E");
    if (Vxc && dV != Vxc) check(cudaMemcpyAsync(Vxc, dV, nn * 8, cudaMemcpyDeviceToHost, s), "copy V");
    if (Eb) check(cudaMemcpyAsync(Eb, w.Eb, nb * 8, cudaMemcpyDeviceToHost, s), "copy Eb");
    if (Nb) check(cudaMemcpyAsync(Nb, w.Nb, nb * 8, cudaMemcpyDeviceToHost, s), "copy Nb");
    check(cudaStreamSynchronize(s), "integrate");
    if (tot[2] != 0.0) return fail(ctx, GBXC_EINVAL, "P contains a NaN or an infinity");
    if (precision == GBXC_MIXED) {
        int werr = 0;
        check(mixed_read_error(w.mixed, &werr, s), "mixed status");
        if (werr) return fail(ctx, GBXC_ETIMEOUT, "a bounded tensor-core pipeline wait expired (code " +
                                                      std::to_string(werr) + ")");
    }
    if (Exc) *Exc = tot[0];
    if (Nel) *Nel = tot[1];
    return GBXC_OK;
}

// ---------------------------------------------------------------------------
// continuous-batching server
// ---------------------------------------------------------------------------
bool server_busy(gbxc_ctx *ctx) {
    Server &S = ctx->srv;
    if (!S.running) return false;
    std::lock_guard<std::mutex> q(S.qmu);
    if (!S.queue.empty()) return true;
    for (auto &r : S.slot_req)
        if (r) return true;
    return false;
}

// Admit the head of the queue if a slot and arena room are free (FIFO, no overtaking).
// Returns true if a request was admitted.  Called by the scheduler thread.
bool server_admit(gbxc_ctx *ctx) {
    Server &S = ctx->srv;
    std::shared_ptr<Request> r;
    int slot = -1;
    {
        std::lock_guard<std::mutex> q(S.qmu);
        if (S.queue.empty()) return false;
        for (int k = 0; k < S.nslots; ++k)
            if (!S.slot_req[k]) {
                slot = k;
                break;
            }
        if (slot < 0) return false;
        r = S.queue.front();
    }
    std::lock_guard<std::recursive_mutex> lk(ctx->mu);
    cudaSetDevice(ctx->device);
    auto fail_req = [&](int code, const std::string &msg) {
        std::lock_guard<std::mutex> q(S.qmu);
        S.queue.pop_front();
        r->status = code;
        r->err = msg;
        r->state = 2;
        r->t_done = std::chrono::steady_clock::now();
        S.cv.notify_all();
        return true;
    };
    try {
        Molecule &m = get_mol(ctx, r->mol);
        if (!m.has_grid) return fail_req(GBXC_ENOTREADY, "molecule has no grid");
        Schedule &Sch = get_schedule(m, r->precision, 0, m.plan.nbatch(), S.slot_budget);
        size_t fp = footprint(m, Sch, r->precision);
        if (fp > S.arena.cap) return fail_req(GBXC_ENOMEM, "request footprint exceeds the serving arena");
        size_t off = 0;
        if (!S.arena.alloc(fp, &off)) return false;       // wait for memory to free up
        size_t nn = (size_t)m.nbf * m.nbf;
        if (2 * nn + 3 > S.pin_cap[slot]) {                // grow this (idle) slot's pinned staging
            cudaStreamSynchronize(S.streams[slot]);
            cudaFreeHost(S.pin[slot]);
            S.pin[slot] = nullptr;
            S.pin_cap[slot] = 0;
            check(cudaMallocHost(&S.pin[slot], (2 * nn + 3) * 8), "pinned staging");
            S.pin_cap[slot] = 2 * nn + 3;
        }
        double *pin = S.pin[slot];
        std::memcpy(pin, r->P.data(), nn * 8);
        Workspace &w = S.slot_ws[slot];
        w = Workspace{};
        w.stream = S.streams[slot];
        carve(w, S.arena.base + off, m, Sch, r->precision, ctx->ws.mixed.encode_fn);
        cudaStream_t st = S.streams[slot];
        check(cudaMemcpyAsync(w.d_P, pin, nn * 8, cudaMemcpyHostToDevice, st), "copy P");
        check(launch_check_finite(w.d_P, (int64_t)nn, w.d_tot + 2, true, st), "check P");
        enqueue(w, m, Sch, w.d_P, r->functional, r->precision, 0, m.plan.nbatch(), w.d_V, false, st, &ctx->prof);
        check(cudaMemcpyAsync(pin + nn, w.d_V, nn * 8, cudaMemcpyDeviceToHost, st), "copy V");
        check(cudaMemcpyAsync(pin + 2 * nn, w.d_tot, 24, cudaMemcpyDeviceToHost, st), "copy E");
        check(cudaEventRecord(S.done_ev[slot], st), "record");
        std::lock_guard<std::mutex> q(S.qmu);
        S.queue.pop_front();
        r->off = off;
        r->bytes = fp;
        r->slot = slot;
        r->state = 1;
        S.slot_req[slot] = r;
        ++S.admitted;
        return true;
    } catch (const ArgError &e) {
        return fail_req(GBXC_EINVAL, e.msg);
    } catch (const CudaFail &e) {
        return fail_req(GBXC_ECUDA, e.msg);
    } catch (const std::exception &e) {
        return fail_req(GBXC_EINVAL, e.what());
    }
}

// Retire finished slots; returns true if any request completed.
bool server_retire(gbxc_ctx *ctx) {
    Server &S = ctx->srv;
    bool any = false;
    for (int k = 0; k < S.nslots; ++k) {
        std::shared_ptr<Request> r;
        {
            std::lock_guard<std::mutex> q(S.qmu);
            r = S.slot_req[k];
        }
        if (!r) continue;
        cudaError_t e = cudaEventQuery(S.done_ev[k]);
        if (e == cudaErrorNotReady) continue;
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        cudaSetDevice(ctx->device);
        Molecule *m = ctx->mols.count(r->mol) ? ctx->mols[r->mol].get() : nullptr;
        size_t nn = m ? (size_t)m->nbf * m->nbf : 0;
        int status = GBXC_OK;
        std::string msg;
        if (e != cudaSuccess) {
            status = GBXC_ECUDA;
            msg = cudaGetErrorString(e);
        } else if (r->precision == GBXC_MIXED) {
            int werr = 0;
            if (mixed_read_error(S.slot_ws[k].mixed, &werr, S.streams[k]) != cudaSuccess || werr) {
                status = GBXC_ETIMEOUT;
                msg = "a bounded tensor-core pipeline wait expired";
            }
        }
        double *pin = S.pin[k];
        if (status == GBXC_OK && pin[2 * nn + 2] != 0.0) {
            status = GBXC_EINVAL;
            msg = "P contains a NaN or an infinity";
        }
        if (status == GBXC_OK) {
            r->V.assign(pin + nn, pin + 2 * nn);
            r->E = pin[2 * nn];
            r->N = pin[2 * nn + 1];
        }
        S.arena.release(r->off, r->bytes);
        std::lock_guard<std::mutex> q(S.qmu);
        r->status = status;
        r->err = msg;
        r->state = 2;
        r->t_done = std::chrono::steady_clock::now();
        r->P.clear();
        r->P.shrink_to_fit();
        S.slot_req[k].reset();
        ++S.completed;
        S.cv.notify_all();
        any = true;
    }
    return any;
}

void server_loop(gbxc_ctx *ctx) {
    Server &S = ctx->srv;
    cudaSetDevice(ctx->device);
    while (!S.stop.load()) {
        bool progress = server_retire(ctx);
        while (server_admit(ctx)) progress = true;
        if (!progress) {
            std::unique_lock<std::mutex> q(S.qmu);
            S.cv.wait_for(q, std::chrono::microseconds(20));
        }
    }
}

void server_stop(gbxc_ctx *ctx) {
    Server &S = ctx->srv;
    if (!S.running) return;
    S.stop = true;
    S.cv.notify_all();
    if (S.thread.joinable()) S.thread.join();
    for (int k = 0; k < S.nslots; ++k) {
        cudaStreamSynchronize(S.streams[k]);
        cudaStreamDestroy(S.streams[k]);
        cudaEventDestroy(S.done_ev[k]);
        cudaFreeHost(S.pin[k]);
    }
    cudaFree(S.arena_mem);
    {
        std::lock_guard<std::mutex> q(S.qmu);
        for (auto &kv : S.tickets)
            if (kv.second->state != 2) {
                kv.second->state = 2;
                kv.second->status = GBXC_ENOTREADY;
                kv.second->err = "server stopped";
            }
        S.cv.notify_all();
    }
    S.streams.clear();
    S.done_ev.clear();
    S.pin.clear();
    S.pin_cap.clear();
    S.slot_req.clear();
    S.slot_ws.clear();
    S.queue.clear();
    S.running = false;
    S.stop = false;
}

}  // namespace

// ---------------------------------------------------------------------------
// kernel-facing helpers shared with the float64 path
// ---------------------------------------------------------------------------
namespace gbxc {
size_t fp64_row_bytes() { return (size_t)8 * TILE * sizeof(double); }

void append_fp64_vtasks(int j, int n, int64_t s0, int64_t s1, std::vector<int> &tasks) {
    const int VB = 64, KS = 16;
    int nblk = (n + VB - 1) / VB;
    for (int64_t k = s0; k < s1; k += KS) {
        int64_t k1 = std::min<int64_t>(k + KS, s1);
        for (int mb = 0; mb < nblk; ++mb)
            for (int nb = 0; nb < nblk; ++nb) {
                tasks.push_back(j);
                tasks.push_back(mb);
                tasks.push_back(nb);
                tasks.push_back((int)k);
                tasks.push_back((int)k1);
            }
    }
}
}  // namespace gbxc

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int gbxc_create(gbxc_ctx **out, int device, size_t scratch_bytes) {
    if (!out) return GBXC_EINVAL;
    *out = nullptr;
    if (device < -1) return GBXC_EINVAL;
    gbxc_ctx *ctx = nullptr;
    if (device == -1) {   // host-only context: planning and plan export, no CUDA calls
        ctx = new (std::nothrow) gbxc_ctx;
        if (!ctx) return GBXC_ENOMEM;
        ctx->device = -1;
        *out = ctx;
        return GBXC_OK;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device >= ndev) {
        cudaGetLastError();
        return GBXC_ECUDA;
    }
    ctx = new (std::nothrow) gbxc_ctx;
    if (!ctx) return GBXC_ENOMEM;
    ctx->device = device;
    ctx->scratch_budget = scratch_bytes;
    ctx->budget_given = scratch_bytes != 0;
    int rc = guarded(ctx, [&] {
        check(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking), "stream");
        ctx->ws.stream = ctx->stream;
        return GBXC_OK;
    });
    if (rc != GBXC_OK) {
        gbxc_destroy(ctx);
        return rc;
    }
    *out = ctx;
    return GBXC_OK;
}

void gbxc_destroy(gbxc_ctx *ctx) {
    if (!ctx) return;
    if (ctx->device < 0) {
        delete ctx;
        return;
    }
    server_stop(ctx);
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &w : ctx->branch_ws) {
        if (w.stream) {
            cudaStreamSynchronize(w.stream);
            cudaStreamDestroy(w.stream);
        }
        free_workspace(w);
    }
    ctx->branch_ws.clear();
    free_group(ctx->group);
    if (ctx->many.exec) cudaGraphExecDestroy(ctx->many.exec);
    if (ctx->many.fork) cudaEventDestroy(ctx->many.fork);
    for (auto e : ctx->many.join) cudaEventDestroy(e);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (auto &kv : ctx->mols) free_molecule(*kv.second);
    ctx->mols.clear();
    free_workspace(ctx->ws);
    ctx->prof.release();
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

// ---------------------------------------------------------------------------
// plan files: the grid and merged batches of a molecule, reloaded without re-planning
// ---------------------------------------------------------------------------
namespace {
constexpr char kPlanMagic[8] = {'G', 'B', 'X', 'C', 'P', 'L', 'A', 'N'};
constexpr uint32_t kPlanVersion = 1;

// FNV-1a over everything the plan depends on: atoms, shells (centres, L, primitives, purity)
uint64_t molecule_hash(const Molecule &m) {
    uint64_t h = 1469598103934665603ull;
    auto mix = [&](const void *p, size_t n) {
        const unsigned char *c = static_cast<const unsigned char *>(p);
        for (size_t i = 0; i < n; ++i) h = (h ^ c[i]) * 1099511628211ull;
    };
    mix(&m.natoms, sizeof(m.natoms));
    mix(m.xyz.data(), m.xyz.size() * sizeof(double));
    mix(&m.nshell, sizeof(m.nshell));
    for (const DevShell &sh : m.shells) {
        mix(sh.c, sizeof(sh.c));
        mix(&sh.L, sizeof(sh.L));
        mix(&sh.nprim, sizeof(sh.nprim));
        mix(&sh.pure, sizeof(sh.pure));
        mix(sh.alpha, sizeof(double) * sh.nprim);
    }
    return h;
}

int finish_grid(gbxc_ctx *ctx, Molecule &m, const gbxc_grid_spec *spec, bool host_only, bool on_device,
                DevPoints &pts, long long *npts_out, int *nbatch_out);

struct PlanHeader {
    char magic[8];
    uint32_t version, reserved;
    uint64_t hash;
    gbxc_grid_spec spec;
    int64_t npts, nbatch, nleaf, nshell_entries;
};
}  // namespace

int gbxc_save_plan(gbxc_ctx *ctx, int mol, const char *path) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(path, "path is NULL");
        Molecule &m = get_mol(ctx, mol);
        if (!m.has_grid) return fail(ctx, GBXC_ENOTREADY, "molecule has no grid");
        const HostPlan &P = m.plan;
        const size_t n = (size_t)P.npts;
        std::vector<double> x(n), y(n), z(n), wq(n);
        std::vector<int> parent(n);
        std::vector<long long> pidx(n);
        int rc = gbxc_export_plan(ctx, mol, x.data(), y.data(), z.data(), wq.data(), nullptr, parent.data(),
                                  pidx.data(), nullptr, nullptr, nullptr);
        if (rc != GBXC_OK) return rc;
        PlanHeader h;
        std::memset(&h, 0, sizeof(h));
        std::memcpy(h.magic, kPlanMagic, 8);
        h.version = kPlanVersion;
        h.hash = molecule_hash(m);
        h.spec = m.spec;
        h.npts = P.npts;
        h.nbatch = P.nbatch();
        h.nleaf = P.nleaf;
        h.nshell_entries = (int64_t)P.shell_idx.size();
        FILE *f = std::fopen(path, "wb");
        if (!f) return fail(ctx, GBXC_EINVAL, std::string("cannot open ") + path + " for writing");
        bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1;
        auto put = [&](const void *p, size_t bytes) { ok = ok && (bytes == 0 || std::fwrite(p, bytes, 1, f) == 1); };
        put(x.data(), n * 8);
        put(y.data(), n * 8);
        put(z.data(), n * 8);
        put(wq.data(), n * 8);
        put(parent.data(), n * 4);
        put(pidx.data(), n * 8);
        put(P.batch_ptr.data(), P.batch_ptr.size() * 8);
        put(P.shell_ptr.data(), P.shell_ptr.size() * 8);
        put(P.shell_idx.data(), P.shell_idx.size() * 4);
        ok = (std::fclose(f) == 0) && ok;
        if (!ok) return fail(ctx, GBXC_EINVAL, std::string("writing ") + path + " failed");
        return GBXC_OK;
    });
}

int gbxc_load_plan(gbxc_ctx *ctx, int mol, const char *path, long long *npts_out, int *nbatch_out) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(path, "path is NULL");
        Molecule &m = get_mol(ctx, mol);
        bool host_only = ctx->device < 0;
        if (server_busy(ctx)) return fail(ctx, GBXC_ENOTREADY, "requests are in flight; wait for them first");
        FILE *f = std::fopen(path, "rb");
        if (!f) return fail(ctx, GBXC_EINVAL, std::string("cannot open ") + path);
        std::unique_ptr<FILE, int (*)(FILE *)> guard(f, std::fclose);
        PlanHeader h;
        if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kPlanMagic, 8) != 0 ||
            h.version != kPlanVersion)
            return fail(ctx, GBXC_EINVAL, "not a plan file of this version");
        if (h.hash != molecule_hash(m)) return fail(ctx, GBXC_EINVAL, "the plan belongs to another molecule or basis");
        REQUIRE(h.npts >= 0 && h.nbatch >= 0 && h.nshell_entries >= 0 && h.npts < (int64_t(1) << 40) &&
                    h.nbatch <= h.npts + 1 && h.nshell_entries <= h.nbatch * (int64_t)m.nshell,
                "corrupt plan sizes");
        const size_t n = (size_t)h.npts, nb = (size_t)h.nbatch;
        HostPlan P;
        P.x.resize(n);
        P.y.resize(n);
        P.z.resize(n);
        P.wq.resize(n);
        P.parent.resize(n);
        P.point_index.resize(n);
        std::vector<int64_t> bptr(nb + 1), sptr(nb + 1);
        std::vector<int> sidx((size_t)h.nshell_entries);
        bool ok = true;
        auto get = [&](void *p, size_t bytes) { ok = ok && (bytes == 0 || std::fread(p, bytes, 1, f) == 1); };
        get(P.x.data(), n * 8);
        get(P.y.data(), n * 8);
        get(P.z.data(), n * 8);
        get(P.wq.data(), n * 8);
        get(P.parent.data(), n * 4);
        get(P.point_index.data(), n * 8);
        get(bptr.data(), (nb + 1) * 8);
        get(sptr.data(), (nb + 1) * 8);
        get(sidx.data(), sidx.size() * 4);
        if (!ok) return fail(ctx, GBXC_EINVAL, "plan file is truncated");
        // validate before anything is replaced
        REQUIRE(bptr[0] == 0 && bptr[nb] == h.npts && sptr[0] == 0 && sptr[nb] == h.nshell_entries,
                "corrupt batch pointers");
        for (size_t j = 0; j < nb; ++j)
            REQUIRE(bptr[j] <= bptr[j + 1] && sptr[j] <= sptr[j + 1], "corrupt batch pointers");
        for (int s : sidx) REQUIRE(s >= 0 && s < m.nshell, "shell index out of range");
        for (size_t i = 0; i < n; ++i)
            REQUIRE(P.parent[i] >= 0 && P.parent[i] < m.natoms && P.point_index[i] >= 0 &&
                        P.point_index[i] < h.npts,
                    "corrupt point data");
        std::vector<std::vector<int>> bshells(nb);
        std::vector<int64_t> bsize(nb);
        for (size_t j = 0; j < nb; ++j) {
            bshells[j].assign(sidx.begin() + sptr[j], sidx.begin() + sptr[j + 1]);
            bsize[j] = bptr[j + 1] - bptr[j];
        }
        batch_metadata((size_t)m.natoms, m.shells, bshells, bsize, P);
        P.nleaf = (int)h.nleaf;
        if (!host_only) {
            check(cudaStreamSynchronize(ctx->stream), "sync");
            if (ctx->many.exec &&
                std::find(ctx->many.mols.begin(), ctx->many.mols.end(), mol) != ctx->many.mols.end()) {
                cudaGraphExecDestroy(ctx->many.exec);
                ctx->many.exec = nullptr;
                ctx->many.mols.clear();
            }
        }
        drop_group_with(ctx, mol);
        free_grid(m);
        m.spec = h.spec;
        m.plan = std::move(P);
        DevPoints none;
        return finish_grid(ctx, m, &m.spec, host_only, false, none, npts_out, nbatch_out);
    });
}

int gbxc_unload(gbxc_ctx *ctx, int mol) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        auto it = ctx->mols.find(mol);
        if (it == ctx->mols.end()) return fail(ctx, GBXC_ENOENT, "unknown molecule id");
        if (server_busy(ctx)) return fail(ctx, GBXC_ENOTREADY, "requests are in flight; wait for them first");
        if (ctx->device >= 0) {
            check(cudaStreamSynchronize(ctx->stream), "sync");
            if (ctx->many.exec &&
                std::find(ctx->many.mols.begin(), ctx->many.mols.end(), mol) != ctx->many.mols.end()) {
                cudaGraphExecDestroy(ctx->many.exec);   // the cached graph reads this molecule's buffers
                ctx->many.exec = nullptr;
                ctx->many.mols.clear();
            }
            drop_group_with(ctx, mol);
            for (auto t = ctx->tuned.begin(); t != ctx->tuned.end();) {
                const std::vector<int> &ids = t->first.first;
                t = std::find(ids.begin(), ids.end(), mol) != ids.end() ? ctx->tuned.erase(t) : std::next(t);
            }
        }
        free_molecule(*it->second);
        ctx->mols.erase(it);
        return GBXC_OK;
    });
}

const char *gbxc_last_error(const gbxc_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int gbxc_load_basis(gbxc_ctx *ctx, int natoms, const double *xyz, const int *Z, int nshell,
                    const int *shell_atom, const int *shell_L, const int *shell_nprim,
                    const double *alpha, const double *coeff, int *mol_out, int *nbf_out) {
    return gbxc_load_basis_pure(ctx, natoms, xyz, Z, nshell, shell_atom, shell_L, shell_nprim, nullptr, alpha,
                                coeff, mol_out, nbf_out);
}

int gbxc_load_basis_pure(gbxc_ctx *ctx, int natoms, const double *xyz, const int *Z, int nshell,
                         const int *shell_atom, const int *shell_L, const int *shell_nprim,
                         const int *shell_pure, const double *alpha, const double *coeff, int *mol_out,
                         int *nbf_out) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(natoms > 0 && xyz && nshell > 0 && shell_atom && shell_L && shell_nprim && alpha &&
                    coeff && mol_out,
                "bad basis arguments");
        auto m = std::make_unique<Molecule>();
        m->natoms = natoms;
        m->xyz.assign(xyz, xyz + 3 * (size_t)natoms);
        if (Z) m->Z.assign(Z, Z + natoms);
        m->nshell = nshell;
        int fofs = 0, prev_atom = -1;
        for (int s = 0; s < nshell; ++s) {
            DevShell sh{};
            int A = shell_atom[s];
            REQUIRE(A >= 0 && A < natoms, "shell atom out of range");
            REQUIRE(A >= prev_atom, "shells must be grouped by atom in ascending order");
            prev_atom = A;
            REQUIRE(shell_L[s] >= 0 && shell_L[s] <= GBXC_MAX_L, "shell L out of range");
            REQUIRE(shell_nprim[s] >= 1 && shell_nprim[s] <= GBXC_MAX_PRIM, "nprim out of range");
            for (int d = 0; d < 3; ++d) sh.c[d] = xyz[3 * A + d];
            sh.L = shell_L[s];
            sh.nprim = shell_nprim[s];
            sh.fofs = fofs;
            sh.pure = (shell_pure && shell_pure[s] && sh.L >= 2) ? 1 : 0;
            for (int k = 0; k < sh.nprim; ++k) {
                sh.alpha[k] = alpha[(size_t)s * GBXC_MAX_PRIM + k];
                sh.coeff[k] = coeff[(size_t)s * GBXC_MAX_PRIM + k];
                REQUIRE(sh.alpha[k] > 0 && std::isfinite(sh.alpha[k]), "exponents must be positive");
                REQUIRE(std::isfinite(sh.coeff[k]), "coefficients must be finite");
            }
            fofs += shell_nfunc(sh);
            m->shells.push_back(sh);
        }
        m->nbf = fofs;
        if (ctx->device < 0) {
            int id = ctx->next_id++;
            *mol_out = id;
            if (nbf_out) *nbf_out = m->nbf;
            ctx->mols[id] = std::move(m);
            return GBXC_OK;
        }
        check(build_mixed_resident(m->shells, m->mixed_res), "double-float shells");
        check(cudaMalloc(&m->d_shells, sizeof(DevShell) * nshell), "cudaMalloc shells");
        check(cudaMemcpy(m->d_shells, m->shells.data(), sizeof(DevShell) * nshell,
                         cudaMemcpyHostToDevice), "upload shells");
        check(cudaMalloc(&m->d_atoms, sizeof(double) * 3 * natoms), "cudaMalloc atoms");
        check(cudaMemcpy(m->d_atoms, xyz, sizeof(double) * 3 * natoms, cudaMemcpyHostToDevice),
              "upload atoms");
        std::vector<double> rnn(natoms, 0.0);
        for (int a = 0; a < natoms; ++a) {
            double best = INFINITY;
            for (int b = 0; b < natoms; ++b) {
                if (a == b) continue;
                double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1],
                       dz = xyz[3 * a + 2] - xyz[3 * b + 2];
                best = std::min(best, std::sqrt(dx * dx + dy * dy + dz * dz));
            }
            rnn[a] = best;
        }
        check(cudaMalloc(&m->d_rnn, sizeof(double) * natoms), "cudaMalloc rnn");
        check(cudaMemcpy(m->d_rnn, rnn.data(), sizeof(double) * natoms, cudaMemcpyHostToDevice),
              "upload rnn");
        // neighbour lists by distance (ties by index) for the SSF screening of the weights
        const size_t nn1 = (size_t)natoms * (size_t)std::max(natoms - 1, 0);
        std::vector<int> nbr(std::max<size_t>(nn1, 1), 0);
        std::vector<double> nbr_r(std::max<size_t>(nn1, 1), 0.0);
        for (int a = 0; a < natoms; ++a) {
            std::vector<std::pair<double, int>> d;
            for (int b = 0; b < natoms; ++b) {
                if (a == b) continue;
                double dx = xyz[3 * a] - xyz[3 * b], dy = xyz[3 * a + 1] - xyz[3 * b + 1],
                       dz = xyz[3 * a + 2] - xyz[3 * b + 2];
                d.emplace_back(std::sqrt(dx * dx + dy * dy + dz * dz), b);
            }
            std::sort(d.begin(), d.end());
            for (size_t k = 0; k < d.size(); ++k) {
                nbr[(size_t)a * (natoms - 1) + k] = d[k].second;
                nbr_r[(size_t)a * (natoms - 1) + k] = d[k].first;
            }
        }
        check(cudaMalloc(&m->d_nbr, sizeof(int) * nbr.size()), "cudaMalloc neighbours");
        check(cudaMemcpy(m->d_nbr, nbr.data(), sizeof(int) * nbr.size(), cudaMemcpyHostToDevice), "upload neighbours");
        check(cudaMalloc(&m->d_nbr_r, sizeof(double) * nbr_r.size()), "cudaMalloc neighbour distances");
        check(cudaMemcpy(m->d_nbr_r, nbr_r.data(), sizeof(double) * nbr_r.size(), cudaMemcpyHostToDevice),
              "upload neighbour distances");
        int id = ctx->next_id++;
        *mol_out = id;
        if (nbf_out) *nbf_out = m->nbf;
        ctx->mols[id] = std::move(m);
        return GBXC_OK;
    });
}

namespace {
int load_grid_impl(gbxc_ctx *ctx, int mol, const gbxc_grid_spec *spec, long long *npts_out, int *nbatch_out,
                   bool on_device);
}

int gbxc_load_grid(gbxc_ctx *ctx, int mol, const gbxc_grid_spec *spec, long long *npts_out,
                   int *nbatch_out) {
    return load_grid_impl(ctx, mol, spec, npts_out, nbatch_out, false);
}

int gbxc_load_grid_device(gbxc_ctx *ctx, int mol, const gbxc_grid_spec *spec, long long *npts_out,
                          int *nbatch_out) {
    return load_grid_impl(ctx, mol, spec, npts_out, nbatch_out, true);
}

namespace {
// The plan of `m` is built (m.plan; device-planned point arrays in *pts when on_device):
// upload it, compute the partition weights on the device, mark the grid loaded.
int finish_grid(gbxc_ctx *ctx, Molecule &m, const gbxc_grid_spec *spec, bool host_only, bool on_device,
                DevPoints &pts, long long *npts_out, int *nbatch_out) {
    m.work = 0.0;
    for (double wj : m.plan.work) m.work += wj;
    if (host_only) {
        m.has_grid = true;
        if (npts_out) *npts_out = (long long)m.plan.npts;
        if (nbatch_out) *nbatch_out = m.plan.nbatch();
        return GBXC_OK;
    }
    cudaStream_t s = ctx->stream;
    HostPlan &P = m.plan;
    if (on_device) {
        m.dev.x = pts.x;
        m.dev.y = pts.y;
        m.dev.z = pts.z;
        m.dev.wq = pts.wq;
        m.dev.parent = pts.parent;
        m.d_point_index = pts.point_index;
    } else {
        m.dev.x = dev_upload(m, P.x, s);
        m.dev.y = dev_upload(m, P.y, s);
        m.dev.z = dev_upload(m, P.z, s);
        m.dev.wq = dev_upload(m, P.wq, s);
        m.dev.parent = dev_upload(m, P.parent, s);
        m.d_point_index = nullptr;
    }
    m.dev.w = dev_alloc<double>(m, P.npts);
    m.dev.shell_ptr = dev_upload(m, P.shell_ptr, s);
    m.dev.shell_idx = dev_upload(m, P.shell_idx, s);
    m.dev.func_ptr = dev_upload(m, P.func_ptr, s);
    m.dev.func_idx = dev_upload(m, P.func_idx, s);
    m.dev.tile_batch = dev_upload(m, P.tile_batch, s);
    m.dev.tile_first = dev_upload(m, P.tile_first, s);
    m.dev.tile_count = dev_upload(m, P.tile_count, s);
    m.dev.tile_row = dev_upload(m, P.tile_row, s);
    m.dev.batch_tile = dev_upload(m, P.batch_tile, s);
    m.dev.batch_ptr = dev_upload(m, P.batch_ptr, s);
    m.d_tileE = dev_alloc<double>(m, P.ntiles());
    m.d_tileN = dev_alloc<double>(m, P.ntiles());
    m.d_Eb = dev_alloc<double>(m, P.nbatch());
    m.d_Nb = dev_alloc<double>(m, P.nbatch());
    WeightsArgs wa;
    wa.x = m.dev.x;
    wa.y = m.dev.y;
    wa.z = m.dev.z;
    wa.wq = m.dev.wq;
    wa.parent = m.dev.parent;
    wa.atoms = m.d_atoms;
    wa.rnn = m.d_rnn;
    wa.nbr = m.d_nbr;
    wa.nbr_r = m.d_nbr_r;
    wa.w = m.dev.w;
    wa.npts = P.npts;
    wa.natoms = m.natoms;
    wa.scheme = spec->partition;
    wa.prof = &ctx->prof;
    check(launch_partition_weights(wa, s), "partition weights");
    check(cudaStreamSynchronize(s), "load_grid");
    m.has_grid = true;
    if (npts_out) *npts_out = (long long)P.npts;
    if (nbatch_out) *nbatch_out = P.nbatch();
    return GBXC_OK;
}

int load_grid_impl(gbxc_ctx *ctx, int mol, const gbxc_grid_spec *spec, long long *npts_out, int *nbatch_out,
                   bool on_device) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(spec, "spec is NULL");
        REQUIRE(spec->angular == GBXC_ANGULAR_PRODUCT || spec->angular == GBXC_ANGULAR_LEBEDEV,
                "unknown angular rule");
        if (spec->angular == GBXC_ANGULAR_LEBEDEV)
            REQUIRE(spec->nrad > 0 && lebedev_supported(spec->ntheta),
                    "no Lebedev rule of that many points (6 14 26 38 50 86 110 146 170 194 302 590 974)");
        else
            REQUIRE(spec->nrad > 0 && spec->ntheta > 0 && spec->nphi > 0, "grid sizes must be positive");
        REQUIRE(spec->partition == GBXC_BECKE || spec->partition == GBXC_SSF, "unknown partition");
        REQUIRE(spec->max_batch > 0, "max_batch must be positive");
        REQUIRE(spec->eta > 0 && spec->eta < 1 && spec->mk_alpha > 0, "bad eta or mk_alpha");
        Molecule &m = get_mol(ctx, mol);
        bool host_only = ctx->device < 0;
        if (server_busy(ctx)) return fail(ctx, GBXC_ENOTREADY, "requests are in flight; wait for them first");
        if (!host_only) check(cudaStreamSynchronize(ctx->stream), "sync");
        if (!host_only && ctx->many.exec) {
            cudaGraphExecDestroy(ctx->many.exec);
            ctx->many.exec = nullptr;
            ctx->many.mols.clear();
        }
        if (on_device) REQUIRE(!host_only, "the device planner needs a device context");
        drop_group_with(ctx, mol);
        free_grid(m);
        m.spec = *spec;
        std::vector<double> x, y, z, wq;
        std::vector<int> parent;
        std::vector<double> rcut(m.nshell);
        for (int s = 0; s < m.nshell; ++s)
            rcut[s] = shell_cutoff(m.shells[s].alpha, m.shells[s].nprim, spec->eta);
        DevPoints pts;
        if (on_device) {
            int status = 0;
            check(device_plan(m.xyz, m.shells, rcut, *spec, m.plan, pts, ctx->stream, &status), "device planner");
            if (status == 1) return fail(ctx, GBXC_EINVAL, "grid too large for the device planner (>= 2^31 points)");
            if (status == 2) return fail(ctx, GBXC_ECUDA, "device planner: cell stack overflow");
            for (void *q : {(void *)pts.x, (void *)pts.y, (void *)pts.z, (void *)pts.wq, (void *)pts.parent,
                            (void *)pts.point_index})
                m.dev_allocs.push_back(q);
        } else {
            build_molecular_grid(m.xyz, *spec, x, y, z, wq, parent);
            build_plan(m.xyz, m.shells, rcut, m.nbf, *spec, x, y, z, wq, parent, m.plan);
        }
        return finish_grid(ctx, m, spec, host_only, on_device, pts, npts_out, nbatch_out);
    });
}

}  // namespace

int gbxc_plan_info_get(gbxc_ctx *ctx, int mol, gbxc_plan_info *info) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(info, "info is NULL");
        Molecule &m = get_mol(ctx, mol);
        std::memset(info, 0, sizeof(*info));
        info->natoms = m.natoms;
        info->nshell = m.nshell;
        info->nbf = m.nbf;
        if (!m.has_grid) return GBXC_OK;
        const HostPlan &P = m.plan;
        info->npts = (long long)P.npts;
        info->nbatch = P.nbatch();
        info->nleaf = P.nleaf;
        info->nshell_entries = (long long)P.shell_idx.size();
        info->nfunc_entries = (long long)P.func_idx.size();
        info->ntiles = (long long)P.ntiles();
        double smn = 0, smn1 = 0, work = 0, sms = 0, sn2 = 0;
        int nmax = 0;
        for (int j = 0; j < P.nbatch(); ++j) {
            double mj = (double)(P.batch_ptr[j + 1] - P.batch_ptr[j]);
            double nj = (double)(P.func_ptr[j + 1] - P.func_ptr[j]);
            smn += mj * nj * nj;
            smn1 += mj * nj;
            sms += mj * (double)(P.shell_ptr[j + 1] - P.shell_ptr[j]);
            sn2 += nj * nj;
            nmax = std::max(nmax, (int)(P.func_ptr[j + 1] - P.func_ptr[j]));
            work += P.work[j];
        }
        info->sum_mn2 = smn;
        info->sum_mn = smn1;
        info->work = work;
        info->sum_ms = sms;
        info->sum_n2 = sn2;
        info->max_nfunc = nmax;
        return GBXC_OK;
    });
}

int gbxc_export_plan(gbxc_ctx *ctx, int mol, double *x, double *y, double *z, double *wq, double *w,
                     int *parent, long long *point_index, long long *batch_ptr,
                     long long *shell_ptr, int *shell_idx) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        Molecule &m = get_mol(ctx, mol);
        if (!m.has_grid) return fail(ctx, GBXC_ENOTREADY, "molecule has no grid");
        const HostPlan &P = m.plan;
        size_t n = (size_t)P.npts;
        if (P.x.size() == n) {
            if (x) std::memcpy(x, P.x.data(), n * 8);
            if (y) std::memcpy(y, P.y.data(), n * 8);
            if (z) std::memcpy(z, P.z.data(), n * 8);
            if (wq) std::memcpy(wq, P.wq.data(), n * 8);
            if (parent) std::memcpy(parent, P.parent.data(), n * 4);
            if (point_index)
                for (size_t i = 0; i < n; ++i) point_index[i] = P.point_index[i];
        } else {   // planned on the device: the point arrays live there only
            if (x) check(cudaMemcpy(x, m.dev.x, n * 8, cudaMemcpyDeviceToHost), "copy x");
            if (y) check(cudaMemcpy(y, m.dev.y, n * 8, cudaMemcpyDeviceToHost), "copy y");
            if (z) check(cudaMemcpy(z, m.dev.z, n * 8, cudaMemcpyDeviceToHost), "copy z");
            if (wq) check(cudaMemcpy(wq, m.dev.wq, n * 8, cudaMemcpyDeviceToHost), "copy wq");
            if (parent) check(cudaMemcpy(parent, m.dev.parent, n * 4, cudaMemcpyDeviceToHost), "copy parent");
            if (point_index)
                check(cudaMemcpy(point_index, m.d_point_index, n * 8, cudaMemcpyDeviceToHost), "copy point index");
        }
        if (batch_ptr)
            for (size_t i = 0; i < P.batch_ptr.size(); ++i) batch_ptr[i] = P.batch_ptr[i];
        if (shell_ptr)
            for (size_t i = 0; i < P.shell_ptr.size(); ++i) shell_ptr[i] = P.shell_ptr[i];
        if (shell_idx) std::memcpy(shell_idx, P.shell_idx.data(), P.shell_idx.size() * 4);
        if (w) {
            REQUIRE(ctx->device >= 0, "partition weights need a device context");
            check(cudaMemcpy(w, m.dev.w, n * 8, cudaMemcpyDeviceToHost), "copy w");
        }
        return GBXC_OK;
    });
}

int gbxc_integrate(gbxc_ctx *ctx, int mol, const double *P, int functional, int precision,
                   double *Exc, double *Vxc, double *Nel, void *stream) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        Molecule &m = get_mol(ctx, mol);
        if (!m.has_grid) return fail(ctx, GBXC_ENOTREADY, "molecule has no grid");
        return integrate_impl(ctx, mol, P, functional, precision, 0, m.plan.nbatch(), Exc, Vxc,
                              Nel, nullptr, nullptr, stream);
    });
}

int gbxc_integrate_uks(gbxc_ctx *ctx, int mol, const double *Pa, const double *Pb, int functional, int precision,
                       double *Exc, double *Va, double *Vb, double *Nel, void *stream) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(ctx->device >= 0, "integration needs a device context");
        Molecule &m = get_mol(ctx, mol);
        if (!m.has_grid) return fail(ctx, GBXC_ENOTREADY, "molecule has no grid");
        REQUIRE(Pa && Pb, "P is NULL");
        for (const void *q : {(const void *)Pa, (const void *)Pb, (const void *)Va, (const void *)Vb})
            REQUIRE(!q || !on_other_device(q, ctx->device), "a buffer is memory of another device");
        REQUIRE(semilocal_lda_gga(functional), "unknown functional");
        REQUIRE(precision == GBXC_FP64 || precision == GBXC_MIXED, "unknown precision");
        const int nb = m.plan.nbatch();
        cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
        const size_t nn = (size_t)m.nbf * m.nbf;
        Workspace &w = ctx->ws;
        const Schedule &S = get_schedule(m, precision, 0, nb, scratch_budget(ctx));
        reserve(w, m, S, precision);
        if (precision == GBXC_MIXED) check(mixed_reserve_uks(w.mixed, S.max_rows, m.nbf), "mixed spin buffers");
        if (nn > w.mat2_cap || !w.d_P2) {
            size_t c0 = w.mat2_cap, c1 = w.mat2_cap, c2 = w.mat2_cap;
            grow_buf(w.d_P2, c0, nn, "P_b");
            grow_buf(w.d_Vacc2, c1, nn, "V_acc_b");
            grow_buf(w.d_V2, c2, nn, "V_b");
            w.mat2_cap = nn;
        }
        const double *dPa = Pa, *dPb = Pb;
        if (!is_device_ptr(Pa)) {
            check(cudaMemcpyAsync(w.d_P, Pa, nn * 8, cudaMemcpyHostToDevice, s), "copy P_a");
            dPa = w.d_P;
        }
        if (!is_device_ptr(Pb)) {
            check(cudaMemcpyAsync(w.d_P2, Pb, nn * 8, cudaMemcpyHostToDevice, s), "copy P_b");
            dPb = w.d_P2;
        }
        check(launch_check_finite(dPa, (int64_t)nn, w.d_tot + 2, true, s), "check P_a");
        check(launch_check_finite(dPb, (int64_t)nn, w.d_tot + 2, false, s), "check P_b");
        double *dVa = (Va && is_device_ptr(Va)) ? Va : w.d_V;
        double *dVb = (Vb && is_device_ptr(Vb)) ? Vb : w.d_V2;
        check(cudaMemsetAsync(w.d_Vacc, 0, nn * 8, s), "zero V_a");
        check(cudaMemsetAsync(w.d_Vacc2, 0, nn * 8, s), "zero V_b");
        if (precision == GBXC_MIXED) check(mixed_begin_uks(w.mixed, dPa, dPb, m.nbf, s), "mixed begin");
        for (size_t ci = 0; ci < S.chunks.size(); ++ci) {
            const auto &c = S.chunks[ci];
            ChunkArgs a;
            a.plan = m.dev;
            a.shells = m.d_shells;
            a.nbf = m.nbf;
            a.t0 = c.t0;
            a.t1 = c.t1;
            a.row0 = c.row0;
            a.rows = c.rows;
            a.max_nfunc = c.max_nfunc;
            a.functional = functional;
            a.P = dPa;
            a.Vacc = w.d_Vacc;
            a.tileE = w.tileE;
            a.tileN = w.tileN;
            a.scratch = w.scratch;
            a.vtasks = S.d_tasks ? S.d_tasks + 5 * c.task0 : nullptr;
            a.nvtasks = (int)c.ntask;
            a.prof = &ctx->prof;
            if (precision == GBXC_FP64)
                check(launch_fp64_chunk_uks(a, dPb, w.d_Vacc2, s), "unrestricted chunk");
            else
                check(launch_mixed_chunk_uks(a, w.mixed, m.mixed_res, S.mixed, (int)ci, w.d_Vacc2, s),
                      "unrestricted mixed chunk");
        }
        FinishArgs f;
        f.Vacc = w.d_Vacc;
        f.V = Va ? dVa : nullptr;
        f.nbf = m.nbf;
        f.tileE = w.tileE;
        f.tileN = w.tileN;
        f.batch_tile = m.dev.batch_tile;
        f.b0 = 0;
        f.b1 = nb;
        f.Eb = w.Eb;
        f.Nb = w.Nb;
        f.tot = w.d_tot;
        f.prof = &ctx->prof;
        check(launch_finish(f, s), "finish");
        if (Vb) check(launch_symmetrize(w.d_Vacc2, dVb, m.nbf, s), "symmetrise V_b");
        double tot[3];
        check(cudaMemcpyAsync(tot, w.d_tot, 24, cudaMemcpyDeviceToHost, s), "copy E");
        if (Va && dVa != Va) check(cudaMemcpyAsync(Va, dVa, nn * 8, cudaMemcpyDeviceToHost, s), "copy V_a");
        if (Vb && dVb != Vb) check(cudaMemcpyAsync(Vb, dVb, nn * 8, cudaMemcpyDeviceToHost, s), "copy V_b");
        check(cudaStreamSynchronize(s), "integrate unrestricted");
        if (tot[2] != 0.0) return fail(ctx, GBXC_EINVAL, "P_a or P_b contains a NaN or an infinity");
        if (precision == GBXC_MIXED) {
            int werr = 0;
            check(mixed_read_error(w.mixed, &werr, s), "mixed status");
            if (werr) return fail(ctx, GBXC_ETIMEOUT, "a bounded tensor-core pipeline wait expired (code " +
                                                          std::to_string(werr) + ")");
        }
        if (Exc) *Exc = tot[0];
        if (Nel) *Nel = tot[1];
        return GBXC_OK;
    });
}

int gbxc_integrate_batches(gbxc_ctx *ctx, int mol, const double *P, int functional, int precision,
                           int batch_begin, int batch_end, double *Exc, double *Vxc, double *Nel,
                           double *E_batch, double *N_batch, void *stream) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        Molecule &m = get_mol(ctx, mol);
        if (!m.has_grid) return fail(ctx, GBXC_ENOTREADY, "molecule has no grid");
        return integrate_impl(ctx, mol, P, functional, precision, batch_begin, batch_end, Exc, Vxc,
                              Nel, E_batch, N_batch, stream);
    });
}

int gbxc_debug_batch(gbxc_ctx *ctx, int mol, int batch, const double *P, int functional, int precision,
                     double *phi, double *gx, double *gy, double *gz, double *z) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(ctx->device >= 0, "needs a device context");
        Molecule &m = get_mol(ctx, mol);
        if (!m.has_grid) return fail(ctx, GBXC_ENOTREADY, "molecule has no grid");
        REQUIRE(batch >= 0 && batch < m.plan.nbatch(), "batch out of range");
        REQUIRE(semilocal_lda_gga(functional), "spin-restricted LDA/GGA only");
        double E, N;
        // the mixed form forms Z inside its slicing kernel; keep_z makes it leave Z in the slab
        struct KeepZ {
            MixedCtx &c;
            explicit KeepZ(MixedCtx &x) : c(x) { c.keep_z = 1; }
            ~KeepZ() { c.keep_z = 0; }
        } keep(ctx->ws.mixed);
        int rc = integrate_impl(ctx, mol, P, functional, precision, batch, batch + 1, &E, nullptr, &N, nullptr,
                                nullptr, nullptr);
        if (rc != GBXC_OK) return rc;
        const Schedule &S = get_schedule(m, precision, batch, batch + 1, scratch_budget(ctx));
        REQUIRE(S.chunks.size() == 1, "the batch does not fit one chunk");
        const Schedule::Chunk &c = S.chunks[0];
        const size_t plane = (size_t)c.rows * TILE;
        std::vector<char> slab((size_t)c.rows * row_bytes(precision));
        check(cudaMemcpy(slab.data(), ctx->ws.scratch, slab.size(), cudaMemcpyDeviceToHost), "copy slabs");
        // value of component comp (0 Phi, 1-3 grad Phi, 4 Z) at slab element e
        auto value = [&](int comp, size_t e) -> double {
            if (precision == GBXC_FP64) {
                const int planes[5] = {0, 1, 2, 3, 5};
                return reinterpret_cast<const double *>(slab.data())[(size_t)planes[comp] * plane + e];
            }
            const MixedSlabOffsets o = mixed_slab_offsets(c.rows);
            auto bf = [](uint16_t b) {
                uint32_t u = (uint32_t)b << 16;
                float f;
                std::memcpy(&f, &u, 4);
                return (double)f;
            };
            if (comp == 0 || comp == 4) {
                const float *f = reinterpret_cast<const float *>(slab.data() + (comp == 0 ? o.phi : o.x));
                return (double)f[2 * e] + (double)f[2 * e + 1];
            }
            const float *h = reinterpret_cast<const float *>(slab.data() + o.ghi);
            const uint16_t *l = reinterpret_cast<const uint16_t *>(slab.data() + o.glo);
            return (double)h[(size_t)(comp - 1) * plane + e] + bf(l[(size_t)(comp - 1) * plane + e]);
        };
        const HostPlan &Pl = m.plan;
        const int64_t n = Pl.func_ptr[batch + 1] - Pl.func_ptr[batch];
        double *outs[5] = {phi, gx, gy, gz, z};
        for (int64_t t = Pl.batch_tile[batch]; t < Pl.batch_tile[batch + 1]; ++t) {
            const int64_t r0 = Pl.tile_row[t] - c.row0;
            for (int i = 0; i < Pl.tile_count[t]; ++i) {
                const int64_t p = Pl.tile_first[t] + i - Pl.batch_ptr[batch];
                for (int64_t mu = 0; mu < n; ++mu)
                    for (int comp = 0; comp < 5; ++comp)
                        if (outs[comp]) outs[comp][p * n + mu] = value(comp, (size_t)(r0 + mu) * TILE + i);
            }
        }
        return GBXC_OK;
    });
}

int gbxc_integrate_fp64_noalloc(gbxc_ctx *ctx, int mol, const double *P, int functional, double *Vxc,
                                double *EN, void *stream) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(ctx->device >= 0, "integration needs a device context");
        REQUIRE(semilocal_lda_gga(functional), "unknown functional");
        REQUIRE(P && Vxc && EN, "P, Vxc and EN must be device pointers");
        REQUIRE(is_device_ptr(P) && is_device_ptr(Vxc) && is_device_ptr(EN),
                "P, Vxc and EN must be device pointers");
        REQUIRE(!on_other_device(P, ctx->device) && !on_other_device(Vxc, ctx->device) &&
                    !on_other_device(EN, ctx->device),
                "P, Vxc and EN must be memory of the context's device");
        Molecule &m = get_mol(ctx, mol);
        if (!m.has_grid) return fail(ctx, GBXC_ENOTREADY, "molecule has no grid");
        void *scratch = nullptr;
        size_t cap = 0;
        double *flag = nullptr;
        check(noalloc_scratch(&scratch, &cap, &flag), "static scratch address");
        const HostPlan &H = m.plan;
        int64_t max_rows = (int64_t)(cap / fp64_row_bytes());
        for (int64_t t = 0; t < H.ntiles(); ++t)
            if (H.tile_row[t + 1] - H.tile_row[t] > max_rows)
                return fail(ctx, GBXC_ENOMEM, "a batch needs more slab rows than the static scratch holds");
        cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
        size_t nn = (size_t)m.nbf * m.nbf;
        check(cudaMemsetAsync(Vxc, 0, nn * 8, s), "zero V");
        check(launch_check_finite(P, (int64_t)nn, flag, true, s), "check P");
        int64_t t = 0, nt = H.ntiles();
        while (t < nt) {
            ChunkArgs a;
            a.plan = m.dev;
            a.shells = m.d_shells;
            a.nbf = m.nbf;
            a.t0 = t;
            a.row0 = H.tile_row[t];
            a.max_nfunc = 0;
            while (t < nt && H.tile_row[t + 1] - a.row0 <= max_rows) {
                int j = H.tile_batch[t];
                a.max_nfunc = std::max(a.max_nfunc, (int)(H.func_ptr[j + 1] - H.func_ptr[j]));
                ++t;
            }
            a.t1 = t;
            a.rows = H.tile_row[t] - a.row0;
            a.functional = functional;
            a.P = P;
            a.Vacc = Vxc;
            a.tileE = m.d_tileE;
            a.tileN = m.d_tileN;
            a.scratch = scratch;
            a.vtasks = nullptr;
            a.nvtasks = 0;
            a.prof = nullptr;
            check(launch_fp64_chunk_noalloc(a, s), "fp64 chunk (static scratch)");
        }
        check(launch_symmetrize_inplace(Vxc, m.nbf, s), "symmetrise");
        Profiler quiet;   // counts only; never records events
        FinishArgs f;
        f.Vacc = nullptr;
        f.V = nullptr;
        f.nbf = m.nbf;
        f.tileE = m.d_tileE;
        f.tileN = m.d_tileN;
        f.batch_tile = m.dev.batch_tile;
        f.b0 = 0;
        f.b1 = H.nbatch();
        f.Eb = m.d_Eb;
        f.Nb = m.d_Nb;
        f.tot = EN;
        f.prof = &quiet;
        check(launch_finish(f, s), "finish");
        check(launch_poison_if_flagged(flag, EN, s), "non-finite P");
        return GBXC_OK;
    });
}

namespace {

// gbxc_integrate_many with an explicit schedule: W graph branches, GEMM N tile `tile_n`.
// Returns the device time of the graph launch in *ms_out (CUDA events on the context stream).
int many_impl(gbxc_ctx *ctx, int nmol, const int *mol_ids, const double *const *P, const int *functional,
              int precision, int W, int tile_n, double *Exc, double *const *Vxc, double *Nel, float *ms_out) {
    REQUIRE(ctx->device >= 0, "integration needs a device context");
    REQUIRE(nmol > 0 && mol_ids && P && functional, "bad molecule list");
    REQUIRE(precision == GBXC_FP64 || precision == GBXC_MIXED, "unknown precision");
    std::vector<Molecule *> ms(nmol);
    for (int k = 0; k < nmol; ++k) {
        ms[k] = &get_mol(ctx, mol_ids[k]);
        if (!ms[k]->has_grid) return fail(ctx, GBXC_ENOTREADY, "a molecule has no grid");
        REQUIRE(semilocal_lda_gga(functional[k]), "unknown functional");
        REQUIRE(P[k], "P is NULL");
        for (int q = 0; q < k; ++q) REQUIRE(mol_ids[q] != mol_ids[k], "a molecule appears twice");
    }
    W = std::max(1, std::min(W, nmol));
    if (precision == GBXC_FP64) tile_n = 128;
    REQUIRE(mixed_tile_supported(tile_n), "unsupported GEMM tile");
    const size_t budget = side_budget(ctx, ctx->many_budget) / W;
    // longest-processing-time assignment of molecules to graph branches by the work
    // estimate of Eq. batch_work (the paper's greedy minimum-load rule, Algorithm 3)
    std::vector<int> order(nmol);
    for (int k = 0; k < nmol; ++k) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ms[a]->work > ms[b]->work; });
    std::vector<double> load(W, 0.0);
    std::vector<std::vector<int>> br(W);
    for (int k : order) {
        int b = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        br[b].push_back(k);
        load[b] += ms[k]->work;
    }
    std::vector<Schedule *> sch(nmol);
    for (int k = 0; k < nmol; ++k)
        sch[k] = &get_schedule(*ms[k], precision, 0, ms[k]->plan.nbatch(), budget, tile_n);
    if ((int)ctx->branch_ws.size() < W) ctx->branch_ws.resize(W);
    for (int b = 0; b < W; ++b) {
        Workspace &w = ctx->branch_ws[b];
        if (!w.stream) check(cudaStreamCreateWithFlags(&w.stream, cudaStreamNonBlocking), "stream");
        for (int k : br[b]) reserve(w, *ms[k], *sch[k], precision);
    }
    for (int k = 0; k < nmol; ++k) {
        Molecule &m = *ms[k];
        size_t nn = (size_t)m.nbf * m.nbf;
        if (nn > m.many_cap || !m.many_P) {
            size_t c0 = m.many_cap, c1 = m.many_cap, c2 = 0;
            grow_buf(m.many_P, c0, nn, "P");
            grow_buf(m.many_V, c1, nn, "V");
            cudaFree(m.many_tot);
            m.many_tot = nullptr;
            grow_buf(m.many_tot, c2, 2, "totals");
            m.many_cap = nn;
        }
    }
    ManyGraph &G = ctx->many;
    std::vector<int> ids(mol_ids, mol_ids + nmol), fns(functional, functional + nmol);
    if (!(G.exec && G.mols == ids && G.fns == fns && G.precision == precision && G.branches == W &&
          G.tile_n == tile_n && G.budget == budget)) {
        if (G.exec) cudaGraphExecDestroy(G.exec);
        G.exec = nullptr;
        if (!G.fork) check(cudaEventCreateWithFlags(&G.fork, cudaEventDisableTiming), "event");
        while ((int)G.join.size() < W) {
            cudaEvent_t e;
            check(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event");
            G.join.push_back(e);
        }
        Profiler quiet;
        cudaStream_t o = ctx->stream;
        check(cudaStreamBeginCapture(o, cudaStreamCaptureModeRelaxed), "begin capture");
        cudaGraph_t graph = nullptr;
        try {
            check(cudaEventRecord(G.fork, o), "fork");
            for (int b = 0; b < W; ++b) check(cudaStreamWaitEvent(ctx->branch_ws[b].stream, G.fork, 0), "fork");
            for (int b = 0; b < W; ++b)
                for (int k : br[b]) {
                    Molecule &m = *ms[k];
                    enqueue(ctx->branch_ws[b], m, *sch[k], m.many_P, functional[k], precision, 0,
                            m.plan.nbatch(), m.many_V, false, ctx->branch_ws[b].stream, &quiet, m.many_tot);
                }
            for (int b = 0; b < W; ++b) {
                check(cudaEventRecord(G.join[b], ctx->branch_ws[b].stream), "join");
                check(cudaStreamWaitEvent(o, G.join[b], 0), "join");
            }
        } catch (...) {
            cudaStreamEndCapture(o, &graph);
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            throw;
        }
        check(cudaStreamEndCapture(o, &graph), "end capture");
        cudaError_t e = cudaGraphInstantiate(&G.exec, graph, 0);
        cudaGraphDestroy(graph);
        check(e, "instantiate graph");
        G.mols = ids;
        G.fns = fns;
        G.precision = precision;
        G.branches = W;
        G.tile_n = tile_n;
        G.budget = budget;
        for (int c = 0; c < GBXC_NKERNEL; ++c) G.launches[c] = quiet.launches[c];
    }
    cudaStream_t o = ctx->stream;
    double *bad_flag = ctx->branch_ws[0].d_tot + 2;
    for (int k = 0; k < nmol; ++k) {
        size_t nn = (size_t)ms[k]->nbf * ms[k]->nbf;
        check(cudaMemcpyAsync(ms[k]->many_P, P[k], nn * 8, cudaMemcpyDefault, o), "copy P");
        check(launch_check_finite(ms[k]->many_P, (int64_t)nn, bad_flag, k == 0, o), "check P");
    }
    long long total = 0;
    for (int c = 0; c < GBXC_NKERNEL; ++c) {
        ctx->prof.launches[c] += G.launches[c];
        total += G.launches[c];
    }
    if (!ctx->ev0) {
        check(cudaEventCreate(&ctx->ev0), "event");
        check(cudaEventCreate(&ctx->ev1), "event");
    }
    ctx->prof.begin(GBXC_K_OTHER, o);
    check(cudaEventRecord(ctx->ev0, o), "event");
    check(cudaGraphLaunch(G.exec, o), "graph launch");
    check(cudaEventRecord(ctx->ev1, o), "event");
    ctx->prof.end(GBXC_K_OTHER, o, 0);
    std::vector<double> tot(2 * (size_t)nmol);
    double bad = 0.0;
    check(cudaMemcpyAsync(&bad, bad_flag, 8, cudaMemcpyDeviceToHost, o), "copy flag");
    for (int k = 0; k < nmol; ++k) {
        size_t nn = (size_t)ms[k]->nbf * ms[k]->nbf;
        check(cudaMemcpyAsync(&tot[2 * k], ms[k]->many_tot, 16, cudaMemcpyDeviceToHost, o), "copy E");
        if (Vxc && Vxc[k]) check(cudaMemcpyAsync(Vxc[k], ms[k]->many_V, nn * 8, cudaMemcpyDefault, o), "copy V");
    }
    check(cudaStreamSynchronize(o), "integrate many");
    (void)total;
    if (bad != 0.0) return fail(ctx, GBXC_EINVAL, "a P contains a NaN or an infinity");
    if (precision == GBXC_MIXED)
        for (int b = 0; b < W; ++b) {
            int werr = 0;
            check(mixed_read_error(ctx->branch_ws[b].mixed, &werr, ctx->branch_ws[b].stream), "status");
            if (werr) return fail(ctx, GBXC_ETIMEOUT, "a bounded tensor-core pipeline wait expired");
        }
    for (int k = 0; k < nmol; ++k) {
        if (Exc) Exc[k] = tot[2 * k];
        if (Nel) Nel[k] = tot[2 * k + 1];
    }
    if (ms_out) check(cudaEventElapsedTime(ms_out, ctx->ev0, ctx->ev1), "event time");
    return GBXC_OK;
}


// The combined plan of a molecule list (host metadata, device copies, shell tables) and the
// batch -> molecule map.
void build_group(gbxc_ctx *ctx, Group &G, const std::vector<Molecule *> &ms) {
    Molecule &g = G.gm;
    HostPlan &H = g.plan;
    cudaStream_t s = ctx->stream;
    H = HostPlan{};
    H.batch_ptr = {0};
    H.shell_ptr = {0};
    H.func_ptr = {0};
    H.batch_tile = {0};
    H.tile_row = {0};
    std::vector<int> batch_mol;
    int64_t pt = 0, t0 = 0, row = 0;
    int sh0 = 0, b0 = 0;
    G.bofs.clear();
    g.shells.clear();
    g.nbf = 0;
    for (size_t k = 0; k < ms.size(); ++k) {
        const Molecule &m = *ms[k];
        const HostPlan &P = m.plan;
        const int nb = P.nbatch();
        const int64_t nt = P.ntiles();
        G.bofs.push_back(b0);
        for (int j = 0; j < nb; ++j) {
            H.batch_ptr.push_back(P.batch_ptr[j + 1] + pt);
            for (int64_t q = P.shell_ptr[j]; q < P.shell_ptr[j + 1]; ++q) H.shell_idx.push_back(P.shell_idx[q] + sh0);
            H.shell_ptr.push_back((int64_t)H.shell_idx.size());
            H.func_idx.insert(H.func_idx.end(), P.func_idx.begin() + P.func_ptr[j], P.func_idx.begin() + P.func_ptr[j + 1]);
            H.func_ptr.push_back((int64_t)H.func_idx.size());
            H.work.push_back(P.work[j]);
            batch_mol.push_back((int)k);
        }
        for (int64_t t = 0; t < nt; ++t) {
            H.tile_batch.push_back(P.tile_batch[t] + b0);
            H.tile_first.push_back(P.tile_first[t] + pt);
            H.tile_count.push_back(P.tile_count[t]);
            H.tile_row.push_back(row + P.tile_row[t + 1]);
        }
        for (int j = 1; j <= nb; ++j) H.batch_tile.push_back(P.batch_tile[j] + t0);
        g.shells.insert(g.shells.end(), m.shells.begin(), m.shells.end());
        g.nbf = std::max(g.nbf, m.nbf);
        H.nleaf += P.nleaf;
        pt += P.npts;
        t0 += nt;
        row += P.tile_row[nt];
        b0 += nb;
        sh0 += (int)m.shells.size();
    }
    G.bofs.push_back(b0);
    H.npts = pt;
    g.nshell = sh0;
    g.natoms = 0;
    // device copies: the points (batch order) and weights of every molecule, the plan arrays
    g.dev.x = dev_alloc<double>(g, pt);
    g.dev.y = dev_alloc<double>(g, pt);
    g.dev.z = dev_alloc<double>(g, pt);
    g.dev.w = dev_alloc<double>(g, pt);
    int64_t o = 0;
    for (Molecule *m : ms) {
        const size_t b = (size_t)m->plan.npts * 8;
        check(cudaMemcpyAsync(g.dev.x + o, m->dev.x, b, cudaMemcpyDeviceToDevice, s), "copy x");
        check(cudaMemcpyAsync(g.dev.y + o, m->dev.y, b, cudaMemcpyDeviceToDevice, s), "copy y");
        check(cudaMemcpyAsync(g.dev.z + o, m->dev.z, b, cudaMemcpyDeviceToDevice, s), "copy z");
        check(cudaMemcpyAsync(g.dev.w + o, m->dev.w, b, cudaMemcpyDeviceToDevice, s), "copy w");
        o += m->plan.npts;
    }
    g.dev.wq = nullptr;
    g.dev.parent = nullptr;
    g.dev.shell_ptr = dev_upload(g, H.shell_ptr, s);
    g.dev.shell_idx = dev_upload(g, H.shell_idx, s);
    g.dev.func_ptr = dev_upload(g, H.func_ptr, s);
    g.dev.func_idx = dev_upload(g, H.func_idx, s);
    g.dev.tile_batch = dev_upload(g, H.tile_batch, s);
    g.dev.tile_first = dev_upload(g, H.tile_first, s);
    g.dev.tile_count = dev_upload(g, H.tile_count, s);
    g.dev.tile_row = dev_upload(g, H.tile_row, s);
    g.dev.batch_tile = dev_upload(g, H.batch_tile, s);
    g.dev.batch_ptr = dev_upload(g, H.batch_ptr, s);
    G.d_batch_mol = nullptr;
    check(cudaMalloc(&G.d_batch_mol, std::max<size_t>(batch_mol.size(), 1) * sizeof(int)), "cudaMalloc batch map");
    check(cudaMemcpyAsync(G.d_batch_mol, batch_mol.data(), batch_mol.size() * sizeof(int), cudaMemcpyHostToDevice, s),
          "upload batch map");
    check(cudaMalloc(&G.d_mols, ms.size() * sizeof(MolRef)), "cudaMalloc molecule table");
    check(cudaMalloc(&g.d_shells, std::max<size_t>(g.shells.size(), 1) * sizeof(DevShell)), "cudaMalloc shells");
    check(cudaMemcpyAsync(g.d_shells, g.shells.data(), g.shells.size() * sizeof(DevShell), cudaMemcpyHostToDevice, s),
          "upload shells");
    check(build_mixed_resident(g.shells, g.mixed_res), "mixed shells");
    check(cudaStreamSynchronize(s), "build group");
    g.has_grid = true;
}

// Queue one grouped integration: per molecule V_acc <- 0 (and P as double-float planes), the
// chunks of the combined plan, then per molecule V = V_acc + V_acc^T and its E, N.
void enqueue_group(Group &G, const std::vector<Molecule *> &ms, const Schedule &S, int precision, cudaStream_t s,
                   Profiler *prof) {
    Workspace &w = G.ws;
    Molecule &g = G.gm;
    for (Molecule *m : ms) {
        check(cudaMemsetAsync(m->many_Vacc, 0, (size_t)m->nbf * m->nbf * 8, s), "zero V");
        if (precision == GBXC_MIXED) check(mixed_prepare_p(m->many_P, m->many_pdf, m->nbf, s), "P planes");
    }
    if (precision == GBXC_MIXED) check(mixed_reset_error(w.mixed, s), "error word");
    for (size_t ci = 0; ci < S.chunks.size(); ++ci) {
        const auto &c = S.chunks[ci];
        ChunkArgs a;
        a.plan = g.dev;
        a.shells = g.d_shells;
        a.nbf = g.nbf;
        a.t0 = c.t0;
        a.t1 = c.t1;
        a.row0 = c.row0;
        a.rows = c.rows;
        a.max_nfunc = c.max_nfunc;
        a.functional = GBXC_PBE;   // unused: every batch takes its molecule's
        a.P = nullptr;
        a.Vacc = nullptr;
        a.tileE = w.tileE;
        a.tileN = w.tileN;
        a.scratch = w.scratch;
        a.vtasks = S.d_tasks ? S.d_tasks + 5 * c.task0 : nullptr;
        a.nvtasks = (int)c.ntask;
        a.prof = prof;
        a.batch_mol = G.d_batch_mol;
        a.mols = G.d_mols;
        if (precision == GBXC_FP64)
            check(launch_fp64_chunk(a, s), "fp64 chunk (grouped)");
        else
            check(launch_mixed_chunk(a, w.mixed, g.mixed_res, S.mixed, (int)ci, s), "mixed chunk (grouped)");
    }
    for (size_t k = 0; k < ms.size(); ++k) {
        Molecule &m = *ms[k];
        FinishArgs f;
        f.Vacc = m.many_Vacc;
        f.V = m.many_V;
        f.nbf = m.nbf;
        f.tileE = w.tileE;
        f.tileN = w.tileN;
        f.batch_tile = g.dev.batch_tile;
        f.b0 = G.bofs[k];
        f.b1 = G.bofs[k + 1];
        f.Eb = w.Eb;
        f.Nb = w.Nb;
        f.tot = m.many_tot;
        f.prof = prof;
        check(launch_finish(f, s), "finish");
    }
}

// gbxc_integrate_many with the grouped schedule (GEMM N tile `tile_n`).  Returns the device
// time of the graph launch in *ms_out (CUDA events on the context stream).
int group_impl(gbxc_ctx *ctx, int nmol, const int *mol_ids, const double *const *P, const int *functional,
               int precision, int tile_n, double *Exc, double *const *Vxc, double *Nel, float *ms_out) {
    REQUIRE(ctx->device >= 0, "integration needs a device context");
    REQUIRE(nmol > 0 && mol_ids && P && functional, "bad molecule list");
    REQUIRE(precision == GBXC_FP64 || precision == GBXC_MIXED, "unknown precision");
    std::vector<Molecule *> ms(nmol);
    for (int k = 0; k < nmol; ++k) {
        ms[k] = &get_mol(ctx, mol_ids[k]);
        if (!ms[k]->has_grid) return fail(ctx, GBXC_ENOTREADY, "a molecule has no grid");
        REQUIRE(semilocal_lda_gga(functional[k]), "unknown functional");
        REQUIRE(P[k], "P is NULL");
        for (int q = 0; q < k; ++q) REQUIRE(mol_ids[q] != mol_ids[k], "a molecule appears twice");
    }
    if (precision == GBXC_FP64) tile_n = 128;
    REQUIRE(mixed_tile_supported(tile_n), "unsupported GEMM tile");
    const size_t budget = side_budget(ctx, ctx->many_budget);
    cudaStream_t o = ctx->stream;
    std::vector<int> ids(mol_ids, mol_ids + nmol);
    // per-molecule buffers: P, V_acc, V, {E, N} and the double-float P planes
    for (int k = 0; k < nmol; ++k) {
        Molecule &m = *ms[k];
        size_t nn = (size_t)m.nbf * m.nbf;
        if (nn > m.many_cap || !m.many_P || !m.many_Vacc || !m.many_pdf) {
            size_t c0 = 0, c1 = 0, c2 = 0, c3 = 0, c4 = 0;
            cudaFree(m.many_P);
            cudaFree(m.many_V);
            cudaFree(m.many_tot);
            cudaFree(m.many_Vacc);
            cudaFree(m.many_pdf);
            m.many_P = m.many_V = m.many_tot = m.many_Vacc = nullptr;
            m.many_pdf = nullptr;
            grow_buf(m.many_P, c0, nn, "P");
            grow_buf(m.many_V, c1, nn, "V");
            grow_buf(m.many_tot, c2, 2, "totals");
            grow_buf(m.many_Vacc, c3, nn, "V_acc");
            grow_buf(m.many_pdf, c4, mixed_pdf_floats(m.nbf), "P planes");
            m.many_cap = nn;
            if (ctx->group) free_group(ctx->group);   // its graph holds the old buffers
        }
    }
    Group *G = ctx->group.get();
    if (!(G && G->mols == ids && G->precision == precision && G->tile_n == tile_n && G->budget == budget)) {
        free_group(ctx->group);
        ctx->group = std::make_unique<Group>();
        G = ctx->group.get();
        build_group(ctx, *G, ms);
        G->mols = ids;
        G->precision = precision;
        G->tile_n = tile_n;
        G->budget = budget;
        Schedule &S = get_schedule(G->gm, precision, 0, G->gm.plan.nbatch(), budget, tile_n);
        G->ws.stream = o;
        reserve(G->ws, G->gm, S, precision);
        G->h_mols.resize(nmol);
        for (int k = 0; k < nmol; ++k) {
            MolRef &r = G->h_mols[k];
            r.P = ms[k]->many_P;
            r.Vacc = ms[k]->many_Vacc;
            r.pdf = reinterpret_cast<const float2 *>(ms[k]->many_pdf);
            r.nbf = ms[k]->nbf;
            r.functional = functional[k];
        }
        Profiler quiet;
        cudaGraph_t graph = nullptr;
        check(cudaStreamBeginCapture(o, cudaStreamCaptureModeRelaxed), "begin capture");
        try {
            enqueue_group(*G, ms, S, precision, o, &quiet);
        } catch (...) {
            cudaStreamEndCapture(o, &graph);
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            throw;
        }
        check(cudaStreamEndCapture(o, &graph), "end capture");
        cudaError_t e = cudaGraphInstantiate(&G->exec, graph, 0);
        cudaGraphDestroy(graph);
        check(e, "instantiate graph");
        for (int c = 0; c < GBXC_NKERNEL; ++c) G->launches[c] = quiet.launches[c];
    }
    // this call's functionals and P (the graph reads both from device memory when it runs)
    for (int k = 0; k < nmol; ++k) G->h_mols[k].functional = functional[k];
    check(cudaMemcpyAsync(G->d_mols, G->h_mols.data(), nmol * sizeof(MolRef), cudaMemcpyHostToDevice, o),
          "molecule table");
    for (int k = 0; k < nmol; ++k) {
        size_t nn = (size_t)ms[k]->nbf * ms[k]->nbf;
        check(cudaMemcpyAsync(ms[k]->many_P, P[k], nn * 8, cudaMemcpyDefault, o), "copy P");
        check(launch_check_finite(ms[k]->many_P, (int64_t)nn, G->ws.d_tot + 2, k == 0, o), "check P");
    }
    for (int c = 0; c < GBXC_NKERNEL; ++c) ctx->prof.launches[c] += G->launches[c];
    if (!ctx->ev0) {
        check(cudaEventCreate(&ctx->ev0), "event");
        check(cudaEventCreate(&ctx->ev1), "event");
    }
    ctx->prof.begin(GBXC_K_OTHER, o);
    check(cudaEventRecord(ctx->ev0, o), "event");
    check(cudaGraphLaunch(G->exec, o), "graph launch");
    check(cudaEventRecord(ctx->ev1, o), "event");
    ctx->prof.end(GBXC_K_OTHER, o, 0);
    std::vector<double> tot(2 * (size_t)nmol);
    double bad = 0.0;
    check(cudaMemcpyAsync(&bad, G->ws.d_tot + 2, 8, cudaMemcpyDeviceToHost, o), "copy flag");
    for (int k = 0; k < nmol; ++k) {
        size_t nn = (size_t)ms[k]->nbf * ms[k]->nbf;
        check(cudaMemcpyAsync(&tot[2 * k], ms[k]->many_tot, 16, cudaMemcpyDeviceToHost, o), "copy E");
        if (Vxc && Vxc[k]) check(cudaMemcpyAsync(Vxc[k], ms[k]->many_V, nn * 8, cudaMemcpyDefault, o), "copy V");
    }
    check(cudaStreamSynchronize(o), "integrate many");
    if (bad != 0.0) return fail(ctx, GBXC_EINVAL, "a P contains a NaN or an infinity");
    if (precision == GBXC_MIXED) {
        int werr = 0;
        check(mixed_read_error(G->ws.mixed, &werr, o), "status");
        if (werr) return fail(ctx, GBXC_ETIMEOUT, "a bounded tensor-core pipeline wait expired");
    }
    for (int k = 0; k < nmol; ++k) {
        if (Exc) Exc[k] = tot[2 * k];
        if (Nel) Nel[k] = tot[2 * k + 1];
    }
    if (ms_out) check(cudaEventElapsedTime(ms_out, ctx->ev0, ctx->ev1), "event time");
    return GBXC_OK;
}

}  // namespace

int gbxc_integrate_many(gbxc_ctx *ctx, int nmol, const int *mol_ids, const double *const *P,
                        const int *functional, int precision, double *Exc, double *const *Vxc, double *Nel) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(nmol > 0 && mol_ids, "bad molecule list");
        int W = 0, tile_n = 128;   // default: the grouped launch
        auto it = ctx->tuned.find({std::vector<int>(mol_ids, mol_ids + nmol), precision});
        if (it != ctx->tuned.end()) {
            W = it->second.first;
            tile_n = it->second.second;
        }
        if (W == 0) return group_impl(ctx, nmol, mol_ids, P, functional, precision, tile_n, Exc, Vxc, Nel, nullptr);
        return many_impl(ctx, nmol, mol_ids, P, functional, precision, W, tile_n, Exc, Vxc,
                         Nel, nullptr);
    });
}

int gbxc_set_schedule(gbxc_ctx *ctx, int nmol, const int *mol_ids, int precision, int branches, int tile_n) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(nmol > 0 && mol_ids, "bad molecule list");
        REQUIRE(precision == GBXC_FP64 || precision == GBXC_MIXED, "unknown precision");
        REQUIRE(branches >= 0 && branches <= 64, "branches must be 0 (grouped) or in 1..64");
        REQUIRE(mixed_tile_supported(tile_n), "tile_n must be 64 or 128");
        ctx->tuned[{std::vector<int>(mol_ids, mol_ids + nmol), precision}] = {branches, tile_n};
        return GBXC_OK;
    });
}

int gbxc_autotune(gbxc_ctx *ctx, int nmol, const int *mol_ids, const double *const *P, const int *functional,
                  int precision, int *branches_out, int *tile_n_out, double *ms_out) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(nmol > 0 && mol_ids, "bad molecule list");
        REQUIRE(precision == GBXC_FP64 || precision == GBXC_MIXED, "unknown precision");
        std::vector<int> Ws = {0};   // 0: the grouped launch; then graph branch counts
        for (int w : {1, 2, 4, 8, 16})
            if (w <= nmol) Ws.push_back(w);
        if (Ws.back() < std::min(nmol, 16)) Ws.push_back(std::min(nmol, 16));
        std::vector<int> tiles = precision == GBXC_MIXED ? std::vector<int>{128, 64} : std::vector<int>{128};
        double best = 1e300;
        int bw = Ws.front(), bt = tiles.front();
        for (int t : tiles)
            for (int w : Ws) {
                float m0 = 0.f, m1 = 0.f, m2 = 0.f;
                auto run = [&](float *ms) {
                    return w == 0 ? group_impl(ctx, nmol, mol_ids, P, functional, precision, t, nullptr, nullptr,
                                               nullptr, ms)
                                  : many_impl(ctx, nmol, mol_ids, P, functional, precision, w, t, nullptr, nullptr,
                                              nullptr, ms);
                };
                int rc = run(&m0);   // capture + first replay
                if (rc != GBXC_OK) return rc;
                rc = run(&m1);
                if (rc != GBXC_OK) return rc;
                rc = run(&m2);
                if (rc != GBXC_OK) return rc;
                const double v = std::min(m1, m2);
                if (v < best) {
                    best = v;
                    bw = w;
                    bt = t;
                }
            }
        ctx->tuned[{std::vector<int>(mol_ids, mol_ids + nmol), precision}] = {bw, bt};
        if (branches_out) *branches_out = bw;
        if (tile_n_out) *tile_n_out = bt;
        if (ms_out) *ms_out = best;
        return GBXC_OK;
    });
}

int gbxc_serve_start(gbxc_ctx *ctx, int nslots, size_t arena_bytes) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(ctx->device >= 0, "serving needs a device context");
        REQUIRE(nslots >= 1 && nslots <= 64, "nslots must be in 1..64");
        Server &S = ctx->srv;
        REQUIRE(!S.running, "the server is already running");
        size_t fixed = 0;
        size_t cap = arena_bytes ? arena_bytes : side_budget(ctx, fixed);
        cudaError_t e = cudaMalloc(&S.arena_mem, cap);
        if (e != cudaSuccess) {
            cudaGetLastError();
            S.arena_mem = nullptr;
            return fail(ctx, GBXC_ENOMEM, "serving arena allocation failed");
        }
        S.arena.init(S.arena_mem, cap);
        S.nslots = nslots;
        S.slot_budget = std::max<size_t>(cap / (size_t)nslots / 2, (size_t)16 << 20);
        S.streams.assign(nslots, nullptr);
        S.done_ev.assign(nslots, nullptr);
        S.pin.assign(nslots, nullptr);
        S.pin_cap.assign(nslots, 0);
        S.slot_req.assign(nslots, nullptr);
        S.slot_ws.assign(nslots, Workspace{});
        for (int k = 0; k < nslots; ++k) {
            check(cudaStreamCreateWithFlags(&S.streams[k], cudaStreamNonBlocking), "stream");
            check(cudaEventCreateWithFlags(&S.done_ev[k], cudaEventDisableTiming), "event");
        }
        check(mixed_init(ctx->ws.mixed), "tensor-map encoder");
        S.admitted = S.completed = 0;
        S.stop = false;
        S.running = true;
        S.thread = std::thread(server_loop, ctx);
        return GBXC_OK;
    });
}

int gbxc_serve_stop(gbxc_ctx *ctx) {
    if (!ctx) return GBXC_EINVAL;
    if (ctx->device < 0) return GBXC_EINVAL;
    server_stop(ctx);   // joins the scheduler: must not hold the context lock here
    return GBXC_OK;
}

int gbxc_submit(gbxc_ctx *ctx, int mol, const double *P, int functional, int precision, long long *ticket) {
    if (!ctx || !P || !ticket) return GBXC_EINVAL;
    Server &S = ctx->srv;
    auto r = std::make_shared<Request>();
    {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        ctx->err.clear();
        if (!S.running) return fail(ctx, GBXC_ENOTREADY, "the server is not running");
        auto it = ctx->mols.find(mol);
        if (it == ctx->mols.end()) return fail(ctx, GBXC_ENOENT, "unknown molecule id");
        if (!it->second->has_grid) return fail(ctx, GBXC_ENOTREADY, "molecule has no grid");
        if (!semilocal_lda_gga(functional)) return fail(ctx, GBXC_EINVAL, "unknown functional");
        if (precision != GBXC_FP64 && precision != GBXC_MIXED) return fail(ctx, GBXC_EINVAL, "unknown precision");
        size_t nn = (size_t)it->second->nbf * it->second->nbf;
        try {
            r->P.assign(P, P + nn);
        } catch (const std::bad_alloc &) {
            return fail(ctx, GBXC_ENOMEM, "host allocation failed");
        }
    }
    r->mol = mol;
    r->functional = functional;
    r->precision = precision;
    r->t_submit = std::chrono::steady_clock::now();
    std::lock_guard<std::mutex> q(S.qmu);
    r->ticket = S.next_ticket++;
    S.tickets[r->ticket] = r;
    S.queue.push_back(r);
    *ticket = r->ticket;
    S.cv.notify_all();
    return GBXC_OK;
}

int gbxc_wait(gbxc_ctx *ctx, long long ticket, double timeout_s, double *Exc, double *Vxc, double *Nel,
              double *latency_s) {
    if (!ctx) return GBXC_EINVAL;
    Server &S = ctx->srv;
    std::unique_lock<std::mutex> q(S.qmu);
    auto it = S.tickets.find(ticket);
    if (it == S.tickets.end()) return GBXC_ENOENT;
    std::shared_ptr<Request> r = it->second;
    auto deadline = std::chrono::steady_clock::now() +
                    std::chrono::microseconds((long long)(std::max(timeout_s, 0.0) * 1e6));
    while (r->state != 2) {
        if (S.cv.wait_until(q, deadline) == std::cv_status::timeout && r->state != 2) return GBXC_ETIMEOUT;
    }
    S.tickets.erase(ticket);
    q.unlock();
    if (r->status != GBXC_OK) {
        std::lock_guard<std::recursive_mutex> lk(ctx->mu);
        ctx->err = r->err;
        return r->status;
    }
    if (Exc) *Exc = r->E;
    if (Nel) *Nel = r->N;
    if (Vxc) std::memcpy(Vxc, r->V.data(), r->V.size() * 8);
    if (latency_s) *latency_s = std::chrono::duration<double>(r->t_done - r->t_submit).count();
    return GBXC_OK;
}

int gbxc_serve_stats(gbxc_ctx *ctx, long long *queued, long long *running, long long *completed,
                     size_t *arena_free, size_t *arena_cap) {
    if (!ctx) return GBXC_EINVAL;
    Server &S = ctx->srv;
    std::lock_guard<std::mutex> q(S.qmu);
    long long run = 0;
    for (auto &r : S.slot_req)
        if (r) ++run;
    if (queued) *queued = (long long)S.queue.size();
    if (running) *running = run;
    if (completed) *completed = S.completed;
    if (arena_free) *arena_free = S.running ? S.arena.free_bytes() : 0;
    if (arena_cap) *arena_cap = S.running ? S.arena.cap : 0;
    return GBXC_OK;
}

int gbxc_profile_enable(gbxc_ctx *ctx, int on) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        ctx->prof.reset();
        ctx->prof.on = on != 0;
        return GBXC_OK;
    });
}

int gbxc_profile_read(gbxc_ctx *ctx, double *ms, long long *launches) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        ctx->prof.collect();
        for (int k = 0; k < GBXC_NKERNEL; ++k) {
            if (ms) ms[k] = ctx->prof.ms[k];
            if (launches) launches[k] = ctx->prof.launches[k];
        }
        return GBXC_OK;
    });
}

}  // extern "C"
