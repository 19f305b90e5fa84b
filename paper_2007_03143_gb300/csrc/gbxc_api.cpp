// C-ABI of the library: context, molecule/basis/grid loading, integration driver.
//
// The driver follows Algorithm 2 on one device: the plan is built once per
// geometry and stays resident (grid points, partition weights, batch lists);
// each integration copies P in (unless it already lives on the device), walks
// the batches in chunks that fit the scratch budget (the paper's
// memory-saturating device subsets), and reduces E, N and V on the device.
#include <algorithm>
#include <cmath>
#include <cstdio>
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

struct Molecule {
    int natoms = 0, nshell = 0, nbf = 0;
    std::vector<double> xyz;
    std::vector<int> Z;
    std::vector<DevShell> shells;
    DevShell *d_shells = nullptr;
    double *d_atoms = nullptr, *d_rnn = nullptr;
    bool has_grid = false;
    gbxc_grid_spec spec{};
    HostPlan plan;
    DevPlan dev;
    std::vector<void *> dev_allocs;
    double *d_tileE = nullptr, *d_tileN = nullptr, *d_Eb = nullptr, *d_Nb = nullptr;
    Schedule sched;
    MixedResident mixed_res;
};

}  // namespace

struct gbxc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t scratch_budget = 0;
    void *scratch = nullptr;
    size_t scratch_cap = 0;
    double *d_P = nullptr, *d_Vacc = nullptr, *d_V = nullptr, *d_tot = nullptr;
    size_t mat_cap = 0;            // elements of the P/V buffers
    std::string err;
    std::map<int, std::unique_ptr<Molecule>> mols;
    int next_id = 0;
    MixedCtx mixed;
    Profiler prof;
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

void free_grid(Molecule &m) {
    for (void *p : m.dev_allocs) cudaFree(p);
    m.dev_allocs.clear();
    free_schedule(m.sched);
    m.dev = DevPlan{};
    m.has_grid = false;
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

Molecule &get_mol(gbxc_ctx *ctx, int mol) {
    auto it = ctx->mols.find(mol);
    if (it == ctx->mols.end()) throw ArgError{"unknown molecule id " + std::to_string(mol)};
    return *it->second;
}

void ensure_matrices(gbxc_ctx *ctx, int nbf) {
    size_t need = (size_t)nbf * nbf;
    if (need <= ctx->mat_cap && ctx->d_P) return;
    cudaFree(ctx->d_P);
    cudaFree(ctx->d_Vacc);
    cudaFree(ctx->d_V);
    ctx->d_P = ctx->d_Vacc = ctx->d_V = nullptr;
    ctx->mat_cap = 0;
    check(cudaMalloc(&ctx->d_P, std::max<size_t>(need, 1) * 8), "cudaMalloc P");
    check(cudaMalloc(&ctx->d_Vacc, std::max<size_t>(need, 1) * 8), "cudaMalloc V_acc");
    check(cudaMalloc(&ctx->d_V, std::max<size_t>(need, 1) * 8), "cudaMalloc V");
    ctx->mat_cap = need;
}

void ensure_scratch(gbxc_ctx *ctx, size_t bytes) {
    if (bytes <= ctx->scratch_cap && ctx->scratch) return;
    cudaFree(ctx->scratch);
    ctx->scratch = nullptr;
    ctx->scratch_cap = 0;
    cudaError_t e = cudaMalloc(&ctx->scratch, std::max<size_t>(bytes, 256));
    if (e != cudaSuccess) {
        cudaGetLastError();
        throw CudaFail{"scratch allocation of " + std::to_string(bytes) + " bytes failed"};
    }
    ctx->scratch_cap = bytes;
}

// The default budget is fixed at the first integration of the context (40% of the
// free device memory then, at most 48 GiB), so schedules stay valid across calls.
size_t scratch_budget(gbxc_ctx *ctx) {
    if (ctx->scratch_budget) return ctx->scratch_budget;
    size_t fr = 0, tot = 0;
    check(cudaMemGetInfo(&fr, &tot), "cudaMemGetInfo");
    size_t b = (size_t)(0.4 * (double)fr);
    ctx->scratch_budget = std::min<size_t>(b, (size_t)48 << 30);
    return ctx->scratch_budget;
}

// Chunks of tiles whose slabs fit the budget, and the V-contraction tasks of each chunk.
void build_schedule(gbxc_ctx *ctx, Molecule &m, int precision, int b0, int b1) {
    Schedule &S = m.sched;
    size_t budget = scratch_budget(ctx);
    if (S.precision == precision && S.b0 == b0 && S.b1 == b1 && S.budget == budget) return;
    free_schedule(S);
    const HostPlan &P = m.plan;
    size_t row_bytes = precision == GBXC_FP64 ? fp64_row_bytes() : mixed_row_bytes();
    int64_t max_rows = (int64_t)(budget / row_bytes);
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
                append_mixed_vtasks(j, n, s0, s1, tasks);
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
        build_mixed_schedule(m.plan, c0, c1, S.mixed);
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
}

int integrate_impl(gbxc_ctx *ctx, int mol, const double *P, int functional, int precision, int b0,
                   int b1, double *Exc, double *Vxc, double *Nel, double *Eb, double *Nb,
                   void *stream) {
    REQUIRE(ctx->device >= 0, "integration needs a device context");
    Molecule &m = get_mol(ctx, mol);
    if (!m.has_grid) throw ArgError{"molecule has no grid (call gbxc_load_grid first)"};
    REQUIRE(P, "P is NULL");
    REQUIRE(functional == GBXC_SLATER || functional == GBXC_PBE, "unknown functional");
    REQUIRE(precision == GBXC_FP64 || precision == GBXC_MIXED, "unknown precision");
    int nb = m.plan.nbatch();
    REQUIRE(0 <= b0 && b0 <= b1 && b1 <= nb, "batch range out of bounds");
    cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
    size_t nn = (size_t)m.nbf * m.nbf;
    ensure_matrices(ctx, m.nbf);
    build_schedule(ctx, m, precision, b0, b1);
    const Schedule &S = m.sched;
    ensure_scratch(ctx, (size_t)S.max_rows * (precision == GBXC_FP64 ? fp64_row_bytes()
                                                                     : mixed_row_bytes()));
    const double *dP = P;
    if (!is_device_ptr(P)) {
        check(cudaMemcpyAsync(ctx->d_P, P, nn * 8, cudaMemcpyHostToDevice, s), "copy P");
        dP = ctx->d_P;
    }
    double *dV = (Vxc && is_device_ptr(Vxc)) ? Vxc : ctx->d_V;
    check(cudaMemsetAsync(ctx->d_Vacc, 0, nn * 8, s), "zero V");
    if (precision == GBXC_MIXED) {
        check(mixed_prepare(ctx->mixed, m.mixed_res, S.mixed, dP, m.nbf, s), "mixed prepare");
    }
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
        a.Vacc = ctx->d_Vacc;
        a.tileE = m.d_tileE;
        a.tileN = m.d_tileN;
        a.scratch = ctx->scratch;
        a.vtasks = S.d_tasks ? S.d_tasks + 5 * c.task0 : nullptr;
        a.nvtasks = (int)c.ntask;
        a.prof = &ctx->prof;
        if (precision == GBXC_FP64)
            check(launch_fp64_chunk(a, s), "fp64 chunk");
        else
            check(launch_mixed_chunk(a, ctx->mixed, m.mixed_res, S.mixed, (int)ci, s), "mixed chunk");
    }
    FinishArgs f;
    f.Vacc = ctx->d_Vacc;
    f.V = Vxc ? dV : nullptr;
    f.nbf = m.nbf;
    f.tileE = m.d_tileE;
    f.tileN = m.d_tileN;
    f.batch_tile = m.dev.batch_tile;
    f.b0 = b0;
    f.b1 = b1;
    f.Eb = m.d_Eb;
    f.Nb = m.d_Nb;
    f.tot = ctx->d_tot;
    f.prof = &ctx->prof;
    if (Eb || Nb) {
        check(cudaMemsetAsync(m.d_Eb, 0, std::max(nb, 1) * 8, s), "zero Eb");
        check(cudaMemsetAsync(m.d_Nb, 0, std::max(nb, 1) * 8, s), "zero Nb");
    }
    check(launch_finish(f, s), "finish");
    double tot[2];
    check(cudaMemcpyAsync(tot, ctx->d_tot, 16, cudaMemcpyDeviceToHost, s), "copy E");
    if (Vxc && dV != Vxc) check(cudaMemcpyAsync(Vxc, dV, nn * 8, cudaMemcpyDeviceToHost, s), "copy V");
    if (Eb) check(cudaMemcpyAsync(Eb, m.d_Eb, nb * 8, cudaMemcpyDeviceToHost, s), "copy Eb");
    if (Nb) check(cudaMemcpyAsync(Nb, m.d_Nb, nb * 8, cudaMemcpyDeviceToHost, s), "copy Nb");
    check(cudaStreamSynchronize(s), "integrate");
    if (precision == GBXC_MIXED) {
        int werr = 0;
        check(mixed_read_error(ctx->mixed, &werr, s), "mixed status");
        if (werr) return fail(ctx, GBXC_ETIMEOUT, "a bounded tensor-core pipeline wait expired (code " +
                                                      std::to_string(werr) + ")");
    }
    if (Exc) *Exc = tot[0];
    if (Nel) *Nel = tot[1];
    return GBXC_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// kernel-facing helpers shared with the float64 path
// ---------------------------------------------------------------------------
namespace gbxc {
size_t fp64_row_bytes() { return (size_t)6 * TILE * sizeof(double); }

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
    int rc = guarded(ctx, [&] {
        check(cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking), "stream");
        check(cudaMalloc(&ctx->d_tot, 16), "cudaMalloc totals");
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
    cudaSetDevice(ctx->device);
    if (ctx->stream) cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->mols) {
        free_grid(*kv.second);
        cudaFree(kv.second->d_shells);
        free_mixed_resident(kv.second->mixed_res);
        cudaFree(kv.second->d_atoms);
        cudaFree(kv.second->d_rnn);
    }
    ctx->mols.clear();
    free_mixed_ctx(ctx->mixed);
    ctx->prof.release();
    cudaFree(ctx->scratch);
    cudaFree(ctx->d_P);
    cudaFree(ctx->d_Vacc);
    cudaFree(ctx->d_V);
    cudaFree(ctx->d_tot);
    if (ctx->stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char *gbxc_last_error(const gbxc_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

int gbxc_load_basis(gbxc_ctx *ctx, int natoms, const double *xyz, const int *Z, int nshell,
                    const int *shell_atom, const int *shell_L, const int *shell_nprim,
                    const double *alpha, const double *coeff, int *mol_out, int *nbf_out) {
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
            for (int k = 0; k < sh.nprim; ++k) {
                sh.alpha[k] = alpha[(size_t)s * GBXC_MAX_PRIM + k];
                sh.coeff[k] = coeff[(size_t)s * GBXC_MAX_PRIM + k];
                REQUIRE(sh.alpha[k] > 0 && std::isfinite(sh.alpha[k]), "exponents must be positive");
                REQUIRE(std::isfinite(sh.coeff[k]), "coefficients must be finite");
            }
            fofs += (sh.L + 1) * (sh.L + 2) / 2;
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
        int id = ctx->next_id++;
        *mol_out = id;
        if (nbf_out) *nbf_out = m->nbf;
        ctx->mols[id] = std::move(m);
        return GBXC_OK;
    });
}

int gbxc_load_grid(gbxc_ctx *ctx, int mol, const gbxc_grid_spec *spec, long long *npts_out,
                   int *nbatch_out) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(spec, "spec is NULL");
        REQUIRE(spec->nrad > 0 && spec->ntheta > 0 && spec->nphi > 0, "grid sizes must be positive");
        REQUIRE(spec->partition == GBXC_BECKE || spec->partition == GBXC_SSF, "unknown partition");
        REQUIRE(spec->max_batch > 0, "max_batch must be positive");
        REQUIRE(spec->eta > 0 && spec->eta < 1 && spec->mk_alpha > 0, "bad eta or mk_alpha");
        Molecule &m = get_mol(ctx, mol);
        bool host_only = ctx->device < 0;
        if (!host_only) check(cudaStreamSynchronize(ctx->stream), "sync");
        free_grid(m);
        m.spec = *spec;
        std::vector<double> x, y, z, wq;
        std::vector<int> parent;
        build_molecular_grid(m.xyz, *spec, x, y, z, wq, parent);
        std::vector<double> rcut(m.nshell);
        for (int s = 0; s < m.nshell; ++s)
            rcut[s] = shell_cutoff(m.shells[s].alpha, m.shells[s].nprim, spec->eta);
        build_plan(m.xyz, m.shells, rcut, m.nbf, *spec, x, y, z, wq, parent, m.plan);
        if (host_only) {
            m.has_grid = true;
            if (npts_out) *npts_out = (long long)m.plan.x.size();
            if (nbatch_out) *nbatch_out = m.plan.nbatch();
            return GBXC_OK;
        }
        cudaStream_t s = ctx->stream;
        HostPlan &P = m.plan;
        m.dev.x = dev_upload(m, P.x, s);
        m.dev.y = dev_upload(m, P.y, s);
        m.dev.z = dev_upload(m, P.z, s);
        m.dev.wq = dev_upload(m, P.wq, s);
        m.dev.parent = dev_upload(m, P.parent, s);
        m.dev.w = dev_alloc<double>(m, P.x.size());
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
        wa.w = m.dev.w;
        wa.npts = (int64_t)P.x.size();
        wa.natoms = m.natoms;
        wa.scheme = spec->partition;
        wa.prof = &ctx->prof;
        check(launch_partition_weights(wa, s), "partition weights");
        check(cudaStreamSynchronize(s), "load_grid");
        m.has_grid = true;
        if (npts_out) *npts_out = (long long)P.x.size();
        if (nbatch_out) *nbatch_out = P.nbatch();
        return GBXC_OK;
    });
}

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
        info->npts = (long long)P.x.size();
        info->nbatch = P.nbatch();
        info->nleaf = P.nleaf;
        info->nshell_entries = (long long)P.shell_idx.size();
        info->nfunc_entries = (long long)P.func_idx.size();
        info->ntiles = (long long)P.ntiles();
        double smn = 0, work = 0;
        for (int j = 0; j < P.nbatch(); ++j) {
            double mj = (double)(P.batch_ptr[j + 1] - P.batch_ptr[j]);
            double nj = (double)(P.func_ptr[j + 1] - P.func_ptr[j]);
            smn += mj * nj * nj;
            work += P.work[j];
        }
        info->sum_mn2 = smn;
        info->work = work;
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
        size_t n = P.x.size();
        if (x) std::memcpy(x, P.x.data(), n * 8);
        if (y) std::memcpy(y, P.y.data(), n * 8);
        if (z) std::memcpy(z, P.z.data(), n * 8);
        if (wq) std::memcpy(wq, P.wq.data(), n * 8);
        if (parent) std::memcpy(parent, P.parent.data(), n * 4);
        if (point_index)
            for (size_t i = 0; i < n; ++i) point_index[i] = P.point_index[i];
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

int gbxc_integrate_fp64_noalloc(gbxc_ctx *ctx, int mol, const double *P, int functional, double *Vxc,
                                double *EN, void *stream) {
    if (!ctx) return GBXC_EINVAL;
    return guarded(ctx, [&] {
        REQUIRE(ctx->device >= 0, "integration needs a device context");
        REQUIRE(functional == GBXC_SLATER || functional == GBXC_PBE, "unknown functional");
        REQUIRE(P && Vxc && EN, "P, Vxc and EN must be device pointers");
        REQUIRE(is_device_ptr(P) && is_device_ptr(Vxc) && is_device_ptr(EN),
                "P, Vxc and EN must be device pointers");
        Molecule &m = get_mol(ctx, mol);
        if (!m.has_grid) return fail(ctx, GBXC_ENOTREADY, "molecule has no grid");
        void *scratch = nullptr;
        size_t cap = 0;
        check(noalloc_scratch(&scratch, &cap), "static scratch address");
        const HostPlan &H = m.plan;
        int64_t max_rows = (int64_t)(cap / fp64_row_bytes());
        for (int64_t t = 0; t < H.ntiles(); ++t)
            if (H.tile_row[t + 1] - H.tile_row[t] > max_rows)
                return fail(ctx, GBXC_ENOMEM, "a batch needs more slab rows than the static scratch holds");
        cudaStream_t s = stream ? (cudaStream_t)stream : ctx->stream;
        size_t nn = (size_t)m.nbf * m.nbf;
        check(cudaMemsetAsync(Vxc, 0, nn * 8, s), "zero V");
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
        return GBXC_OK;
    });
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
