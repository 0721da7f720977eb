// Host runtime and C ABI of libmhdbunch.so (declared in include/mhd_bunch.h).
//
// Owns the device patch table, the owner map used by the guard fill, the tile lists of
// every compiled kernel configuration, the small work buffers (CFL partial maxima, work
// counters, error word) and the CUDA graph.  The state buffers and the stream belong to
// the caller.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <new>
#include <numeric>
#include <sstream>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/mhd_bunch.h"
#include "mhd_launch.h"
#include "mhd_sched.cuh"
#include "mhd_xfer.cuh"

using namespace mhd;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
    g_err = msg;
    return code;
}

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(MHD_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// smallest of n per-chunk time steps into *out (one warp)
__global__ void min_dt_kernel(const double* __restrict__ v, int n, double* __restrict__ out) {
    double m = v[0];
    for (int i = threadIdx.x; i < n; i += 32) m = fmin(m, v[i]);
    for (int o = 16; o > 0; o >>= 1) m = fmin(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) *out = m;
}

// degenerate-star threshold of the HLLD solver, relative to Bn^2, per precision
double hlld_eps(int rb) { return rb == 8 ? 1e-12 : 1e-6; }

}  // namespace

namespace mhd {
// lets other translation units of the library report through mhd_last_error()
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace mhd

struct mhd_bunch {
    int rb = 4, guard = 3, npatch = 0, ndim = 3;
    std::vector<int> pn;                 // 3 * npatch
    bool have_geom = false;
    double dx[3] = {1, 1, 1};
    std::vector<int64_t> origin;
    int64_t domain[3] = {1, 1, 1};
    int bc[6] = {0, 0, 0, 0, 0, 0};
    double gamma = 5.0 / 3.0, courant = 0.8;
    int limiter = 0;
    int riemann = MHD_RIEMANN_HLLD;
    std::vector<int64_t> offs;
    size_t state_bytes = 0;
    std::vector<PatchDev> hp;
    PatchDev* d_patches = nullptr;
    int* d_owner = nullptr;
    FillGeom fg{};
    // neighbour offsets [npatch][27] of the table-driven guard fill (equal patches on a
    // regular grid only; null otherwise)
    int64_t* d_nboff = nullptr;
    void* d_partial_fc = nullptr;        // per-plane partial maxima of the fused fill + CFL
    // tiles of each step configuration: natural (per patch) order and cost-sorted order
    struct Tiles {
        int4* d_nat = nullptr;
        int4* d_lpt = nullptr;
        int n = 0;
        std::vector<int4> nat_h;             // host copy of the natural order
        std::vector<int> first, count;   // per patch, in natural order
    };
    std::vector<Tiles> tiles;
    std::vector<int> cfg_index;          // compiled configs usable for this ndim
    int* d_work = nullptr;               // 2 ints (persistent work counter, finished CTAs)
    void* d_partial = nullptr;           // CFL partial maxima
    unsigned* d_counter = nullptr;       // CFL last-block counter
    int cfl_grid = 0;
    double* d_dt = nullptr;              // dt of the host-dt entry points
    double* d_dts = nullptr;             // dt per step of advance_host
    int d_dts_cap = 0;
    unsigned* d_err = nullptr;
    void* d_adjF = nullptr;              // adjoint work arrays (allocated on first use)
    void* d_adjG = nullptr;
    void* d_adjU = nullptr;
    void* buf[2] = {nullptr, nullptr};
    int cur = 0;                         // index of the buffer holding U^n
    cudaStream_t stream = nullptr;
    // asynchronous stepping: neighbour lists (owners of each patch's guard zone), per-patch
    // times and slices, device mirrors, and the record of the last run's rounds
    std::vector<std::vector<int>> nbrs;
    std::vector<int> owner_h;
    int64_t ob_bs[3] = {1, 1, 1}, ob_M[3] = {1, 1, 1};
    int* d_slice = nullptr;
    double* d_told = nullptr;
    double* d_tcur = nullptr;
    double* d_dtp = nullptr;
    int4* d_atiles = nullptr;
    int atiles_cap = 0;
    // device scheduler: neighbour lists (CSR), tile index of the chosen configuration, the
    // record of a batch of rounds (list, dt, arrival flag, count per round), tile count,
    // abort flag
    int* d_nb_off = nullptr;
    int* d_nb_idx = nullptr;
    int* d_tfirst = nullptr;
    int* d_tcount = nullptr;
    int* d_rows_list = nullptr;
    double* d_rows_dt = nullptr;
    unsigned char* d_rows_last = nullptr;
    int* d_rows_n = nullptr;
    int* d_ntiles = nullptr;
    unsigned* d_abort = nullptr;
    int* d_ready = nullptr;                 // readiness flag per patch
    unsigned long long* d_rmax = nullptr;   // maximum CFL rate per patch (double bits)
    std::vector<std::vector<int>> log_patches;
    std::vector<std::vector<double>> log_dts;
    // interior layout (host transfers of owned cells only): per-patch offsets, device copy
    // of them, and the device staging buffer of one whole interior state
    std::vector<int64_t> ioff_h;
    int64_t* d_ioff = nullptr;
    void* d_interior = nullptr;
    // host-streamed advance: library-owned copy streams and per-chunk events
    cudaStream_t s_in = nullptr, s_out = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_step, ev_out;
    int mode = MHD_MODE_PERSISTENT, config = -1;
    // MHD_MODE_MIXED: per configuration, the tiles (longest first) of the patches whose
    // size class was assigned that configuration by the autotuner (empty: not assigned)
    struct MixedTiles {
        int4* d_tiles = nullptr;
        int n = 0;
    };
    std::vector<MixedTiles> mixed;
    // MHD_MODE_BUNCH_LISTS: the bunches of mhd_bunch_set_bunches (patch lists) and, per
    // configuration, their tiles (each bunch's tiles longest first, bunches in list order)
    std::vector<int> bunch_patches, bunch_start;
    struct BunchTiles {
        int4* d_tiles = nullptr;
        std::vector<int> first, count;       // per bunch
    };
    std::vector<BunchTiles> btiles;
    // slab of a z-layer decomposition (mhd_bunch_set_slab): the handle owns layers
    // [slab_z0, slab_z1) of the box's patch grid, stored in slots 0..L-1 of the state, and
    // two halo layers (the layer below in slot L, the layer above in slot L+1) that the
    // caller fills (mhd_bunch_slab_unpack) from its neighbours before each guard fill
    bool slab = false;
    int slab_z0 = 0, slab_z1 = 0, slab_nl = 0;
    int64_t slab_ppl = 0;
    PatchDev* d_slab_slots = nullptr;    // [(L+2) * ppl]: every patch slot, for the layer copies
    int64_t* d_slab_ioff = nullptr;      // [ppl]: interior-layout offsets within one layer
    // captured step sequences; with an odd step count the second starts from the other buffer
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    int graph_steps = 0, graph_start = 0;
    int64_t launches = 0;
    int nsm = 0;
    const PrecisionKernels* K = nullptr;
};

namespace {

bool active(const mhd_bunch* b, int d) { return b->domain[d] > 1; }

int default_config(const mhd_bunch* b) {
    // first compiled configuration for this dimensionality
    return b->cfg_index.empty() ? -1 : 0;
}

const StepLaunch& step_cfg(const mhd_bunch* b, int k) { return b->K->step[b->cfg_index[k]]; }

void free_mixed(mhd_bunch* b) {
    for (auto& m : b->mixed) cudaFree(m.d_tiles);
    b->mixed.clear();
}

void free_btiles(mhd_bunch* b) {
    for (auto& t : b->btiles) cudaFree(t.d_tiles);
    b->btiles.clear();
}

void free_tiles(mhd_bunch* b) {
    for (auto& t : b->tiles) {
        cudaFree(t.d_nat);
        cudaFree(t.d_lpt);
    }
    b->tiles.clear();
    free_mixed(b);
    free_btiles(b);
    b->bunch_patches.clear();
    b->bunch_start.clear();
}

void release_graph(mhd_bunch* b) {
    for (int k = 0; k < 2; ++k) {
        if (b->gexec[k]) cudaGraphExecDestroy(b->gexec[k]);
        if (b->graph[k]) cudaGraphDestroy(b->graph[k]);
        b->gexec[k] = nullptr;
        b->graph[k] = nullptr;
    }
    b->graph_steps = 0;
}

int common_create(const int32_t* pn, int npatch, int guard, int nvar, int rb, mhd_bunch** out) {
    if (!out) return fail(MHD_EINVAL, "out is NULL");
    *out = nullptr;
    if (nvar != 8) return fail(MHD_EINVAL, "nvar must be 8 (rho, 3 momenta, E, 3 face fields)");
    if (rb != 4 && rb != 8) return fail(MHD_EINVAL, "real_bytes must be 4 or 8");
    if (guard < 3) return fail(MHD_EINVAL, "guard must be >= 3");
    if (npatch <= 0 || !pn) return fail(MHD_EINVAL, "npatch must be positive");
    // dimensionality from the first patch; all patches must agree on which axes are active
    int act[3];
    for (int d = 0; d < 3; ++d) act[d] = pn[d] > 1;
    int ndim = act[2] ? 3 : (act[1] ? 2 : 1);
    if ((act[2] && !act[1]) || (act[1] && !act[0]) || !act[0])
        return fail(MHD_EINVAL, "active axes must be x, x-y or x-y-z");
    for (int p = 0; p < npatch; ++p)
        for (int d = 0; d < 3; ++d) {
            if (pn[3 * p + d] < 1) return fail(MHD_EINVAL, "patch sizes must be >= 1");
            if ((pn[3 * p + d] > 1) != (act[d] != 0))
                return fail(MHD_EINVAL, "all patches must share the collapsed axes");
            if (pn[3 * p + d] > 4096) return fail(MHD_EINVAL, "patch extent too large");
        }
    mhd_bunch* b = new (std::nothrow) mhd_bunch();
    if (!b) return fail(MHD_ENOMEM, "host allocation failed");
    b->rb = rb;
    b->guard = guard;
    b->npatch = npatch;
    b->ndim = ndim;
    b->pn.assign(pn, pn + 3 * npatch);
    b->K = rb == 4 ? &kernels_f32() : &kernels_f64();
    for (int k = 0; k < b->K->nstep; ++k)
        if (b->K->step[k].ndim == ndim) b->cfg_index.push_back(k);
    // layout
    b->offs.resize(npatch);
    int64_t off = 0;
    b->hp.resize(npatch);
    for (int p = 0; p < npatch; ++p) {
        PatchDev& q = b->hp[p];
        q.nx = pn[3 * p];
        q.ny = pn[3 * p + 1];
        q.nz = pn[3 * p + 2];
        q.gx = act[0] ? guard : 0;
        q.gy = act[1] ? guard : 0;
        q.gz = act[2] ? guard : 0;
        q.X = q.nx + 2 * q.gx;
        q.Y = q.ny + 2 * q.gy;
        q.Z = q.nz + 2 * q.gz;
        q.off = off;
        q.ox = q.oy = q.oz = 0;
        q.clamp = 0;
        b->offs[p] = off;
        off += 8LL * q.X * q.Y * q.Z;
        // keep every patch 16-byte aligned
        const int64_t al = 16 / rb;
        off = (off + al - 1) / al * al;
    }
    b->state_bytes = (size_t)off * rb;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete b;
        return fail(MHD_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
    }
    e = b->K->prepare_fill_cfl();
    if (e != cudaSuccess) {
        delete b;
        return fail(MHD_ECUDA, std::string("kernel attribute: ") + cudaGetErrorString(e));
    }
    for (int k : b->cfg_index) {
        e = b->K->step[k].prepare();
        if (e != cudaSuccess) {
            delete b;
            return fail(MHD_ECUDA, std::string("kernel attribute: ") + cudaGetErrorString(e));
        }
    }
    b->cfl_grid = std::min(npatch, b->nsm * 8);
    e = cudaMalloc(&b->d_patches, sizeof(PatchDev) * npatch);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_work, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_partial, (size_t)b->cfl_grid * rb);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_dt, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_err, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_work, 0, 2 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->d_counter, 0, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, sizeof(unsigned));
    if (e != cudaSuccess) {
        mhd_bunch_destroy(b);
        return fail(MHD_ENOMEM, std::string("device allocation: ") + cudaGetErrorString(e));
    }
    *out = b;
    return MHD_OK;
}

int64_t gcd64(int64_t a, int64_t b) { return b == 0 ? a : gcd64(b, a % b); }

int build_tiles(mhd_bunch* b) {
    free_tiles(b);
    b->tiles.resize(b->cfg_index.size());
    for (size_t k = 0; k < b->cfg_index.size(); ++k) {
        const StepLaunch& L = step_cfg(b, (int)k);
        std::vector<int4> nat;
        auto& T = b->tiles[k];
        T.first.resize(b->npatch);
        T.count.resize(b->npatch);
        for (int p = 0; p < b->npatch; ++p) {
            T.first[p] = (int)nat.size();
            const int nx = b->pn[3 * p], ny = b->pn[3 * p + 1], nz = b->pn[3 * p + 2];
            for (int y0 = 0; y0 < (b->ndim >= 2 ? ny : 1); y0 += (b->ndim >= 2 ? L.ty : 1))
                for (int x0 = 0; x0 < nx; x0 += L.tx) {
                    const int w = std::min(L.tx, nx - x0) * (b->ndim >= 2 ? std::min(L.ty, ny - y0) : 1);
                    nat.push_back(make_int4(p, x0, y0, w * nz));
                }
            T.count[p] = (int)nat.size() - T.first[p];
        }
        std::vector<int4> lpt = nat;
        T.nat_h = nat;
        std::stable_sort(lpt.begin(), lpt.end(), [](const int4& a, const int4& c) { return a.w > c.w; });
        T.n = (int)nat.size();
        CK(cudaMalloc(&T.d_nat, sizeof(int4) * T.n));
        CK(cudaMalloc(&T.d_lpt, sizeof(int4) * T.n));
        CK(cudaMemcpy(T.d_nat, nat.data(), sizeof(int4) * T.n, cudaMemcpyHostToDevice));
        CK(cudaMemcpy(T.d_lpt, lpt.data(), sizeof(int4) * T.n, cudaMemcpyHostToDevice));
    }
    return MHD_OK;
}

StepHostArgs step_args(mhd_bunch* b, const double* dt_ptr, double dt_val) {
    StepHostArgs a;
    a.U = b->buf[b->cur];
    a.Unew = b->buf[1 - b->cur];
    a.slice = nullptr;
    a.dt_patch = nullptr;
    a.patches = b->d_patches;
    a.tiles = nullptr;
    a.ntiles = 0;
    a.ntiles_dev = nullptr;
    a.dynamic = 0;
    a.work = b->d_work;
    a.dt_ptr = dt_ptr;
    a.dt_val = dt_val;
    a.gamma = b->gamma;
    a.eps = hlld_eps(b->rb);
    for (int d = 0; d < 3; ++d) a.dxi[d] = 1.0 / b->dx[d];
    a.limiter = b->limiter;
    a.riemann = b->riemann;
    a.err = b->d_err;
    return a;
}

int not_slab(const mhd_bunch* b) {
    if (b->slab) return fail(MHD_EINVAL, "not available on a slab handle (mhd_bunch_set_slab)");
    return MHD_OK;
}

int ready(const mhd_bunch* b) {
    if (!b) return fail(MHD_EINVAL, "handle is NULL");
    if (!b->have_geom) return fail(MHD_ESTATE, "mhd_bunch_set_geometry has not been called");
    if (!b->buf[0] || !b->buf[1]) return fail(MHD_ESTATE, "mhd_bunch_bind has not been called");
    return MHD_OK;
}

int do_fill(mhd_bunch* b) {
    CK(b->K->fill(b->buf[b->cur], b->d_patches, b->npatch, b->fg, b->d_nboff, b->hp[0].Z, b->d_err, b->stream));
    b->launches++;
    return MHD_OK;
}

// Neighbour table of the table-driven guard fill, for bunches of equal patches (each at
// least `guard` cells on active axes) whose origins lie on the grid of the patch extent:
// for every patch and direction s in {-1,0,1}^3 the state offset of the patch owning the
// cell origin + s * n, wrapped periodically into the box.  Entries of directions that
// cross an outflow box face are never read (the fill clamps there instead); a collapsed
// axis only has s = 0 (other entries hold the patch itself).  Empty when the geometry does
// not qualify (the owner-map fill is used then).
std::vector<int64_t> neighbour_table(const mhd_bunch* b, const int64_t* origin, const int64_t* N,
                                     const std::vector<int>& owner, const int64_t* bs, const int64_t* M) {
    std::vector<int64_t> t;
    const int n[3] = {b->pn[0], b->pn[1], b->pn[2]};
    for (int p = 0; p < b->npatch; ++p)
        for (int d = 0; d < 3; ++d) {
            if (b->pn[3 * p + d] != n[d]) return t;
            if (n[d] > 1 && (n[d] < b->guard || origin[3 * p + d] % n[d] != 0 || N[d] % n[d] != 0)) return t;
        }
    t.assign((size_t)b->npatch * 27, 0);
    for (int p = 0; p < b->npatch; ++p)
        for (int sz = -1; sz <= 1; ++sz)
            for (int sy = -1; sy <= 1; ++sy)
                for (int sx = -1; sx <= 1; ++sx) {
                    const int s[3] = {sx, sy, sz};
                    int64_t c[3];
                    bool used = true;
                    for (int d = 0; d < 3; ++d) {
                        if (n[d] == 1 && s[d] != 0) used = false;
                        c[d] = origin[3 * p + d] + (int64_t)s[d] * n[d];
                        if (c[d] < 0) c[d] += N[d];
                        else if (c[d] >= N[d]) c[d] -= N[d];
                    }
                    int q = p;
                    if (used) q = owner[(size_t)(((c[2] / bs[2]) * M[1] + c[1] / bs[1]) * M[0] + c[0] / bs[0])];
                    t[(size_t)p * 27 + (sz + 1) * 9 + (sy + 1) * 3 + (sx + 1)] = b->offs[q];
                }
    return t;
}

int do_cfl(mhd_bunch* b, double* dt_dev) {
    double dxi[3];
    int act[3];
    for (int d = 0; d < 3; ++d) {
        dxi[d] = 1.0 / b->dx[d];
        act[d] = active(b, d);
    }
    CK(b->K->cfl(b->buf[b->cur], b->d_patches, b->npatch, b->gamma, b->courant, dxi, act, b->d_partial,
                 b->cfl_grid, b->d_counter, dt_dev, b->d_err, b->stream));
    b->launches++;
    return MHD_OK;
}

// guard fill then CFL dt: one fused pass on regular grids, else the two kernels
int do_fill_cfl(mhd_bunch* b, double* dt_dev) {
    if (!b->d_nboff) {
        int rc = do_fill(b);
        return rc ? rc : do_cfl(b, dt_dev);
    }
    double dxi[3];
    int act[3];
    for (int d = 0; d < 3; ++d) {
        dxi[d] = 1.0 / b->dx[d];
        act[d] = active(b, d);
    }
    CK(b->K->fill_cfl(b->buf[b->cur], b->d_patches, b->hp[0], b->npatch, b->d_nboff, b->hp[0].Z, b->gamma, b->courant,
                      dxi, act, b->d_partial_fc, b->d_counter, dt_dev, b->d_err, b->stream));
    b->launches++;
    return MHD_OK;
}

int do_step(mhd_bunch* b, const double* dt_ptr, double dt_val) {
    if (b->cfg_index.empty()) return fail(MHD_EINVAL, "no compiled kernel for this dimensionality");
    const int k = b->config < 0 ? default_config(b) : b->config;
    const StepLaunch& L = step_cfg(b, k);
    const auto& T = b->tiles[k];
    StepHostArgs a = step_args(b, dt_ptr, dt_val);
    if (b->mode == MHD_MODE_PER_PATCH) {
        for (int p = 0; p < b->npatch; ++p) {
            a.tiles = T.d_nat + T.first[p];
            a.ntiles = T.count[p];
            a.dynamic = 0;
            CK(L.launch(&a, T.count[p], b->stream));
            b->launches++;
        }
    } else if (b->mode == MHD_MODE_BUNCHED) {
        a.tiles = T.d_nat;
        a.ntiles = T.n;
        a.dynamic = 0;
        CK(L.launch(&a, T.n, b->stream));
        b->launches++;
    } else if (b->mode == MHD_MODE_BUNCH_LISTS) {
        // one persistent launch per bunch, in list order (each resets the work counter when
        // its last CTA finishes, so the next one starts from zero)
        if (b->btiles.empty()) return fail(MHD_ESTATE, "no bunch lists set (mhd_bunch_set_bunches)");
        const auto& BT = b->btiles[k];
        int occ = 1;
        CK(L.occupancy(&occ));
        occ = std::max(occ, 1);
        for (size_t q = 0; q < BT.count.size(); ++q) {
            a.tiles = BT.d_tiles + BT.first[q];
            a.ntiles = BT.count[q];
            a.dynamic = 1;
            CK(L.launch(&a, std::min(BT.count[q], b->nsm * occ), b->stream));
            b->launches++;
        }
    } else if (b->mode == MHD_MODE_MIXED && !b->mixed.empty()) {
        // one persistent launch per configuration in use (each resets the work counter
        // when its last CTA finishes, so the next one starts from zero)
        for (size_t c = 0; c < b->mixed.size(); ++c) {
            const auto& M = b->mixed[c];
            if (M.n == 0) continue;
            const StepLaunch& Lc = step_cfg(b, (int)c);
            int occ = 1;
            CK(Lc.occupancy(&occ));
            occ = std::max(occ, 1);
            a.tiles = M.d_tiles;
            a.ntiles = M.n;
            a.dynamic = 1;
            CK(Lc.launch(&a, std::min(M.n, b->nsm * occ), b->stream));
            b->launches++;
        }
    } else {
        int occ = 1;
        CK(L.occupancy(&occ));
        occ = std::max(occ, 1);
        const int grid = std::min(T.n, b->nsm * occ);
        a.tiles = T.d_lpt;
        a.ntiles = T.n;
        a.dynamic = 1;
        CK(L.launch(&a, grid, b->stream));
        b->launches++;
    }
    b->cur = 1 - b->cur;
    return MHD_OK;
}

// Tiles (configuration c, longest first) of the patches for which sel(p) holds.
std::vector<int4> class_tiles(const mhd_bunch* b, int c, const std::vector<char>& sel) {
    const auto& T = b->tiles[c];
    std::vector<int4> out;
    for (int p = 0; p < b->npatch; ++p)
        if (sel[p]) out.insert(out.end(), T.nat_h.begin() + T.first[p], T.nat_h.begin() + T.first[p] + T.count[p]);
    std::stable_sort(out.begin(), out.end(), [](const int4& x, const int4& y) { return x.w > y.w; });
    return out;
}

// MHD_MODE_MIXED autotuning: every patch-size class timed with every configuration (a
// persistent launch over the class's tiles at dt = 0, two warm-up and four timed), each
// class assigned its fastest; then the per-configuration tile lists.  The caller saves and
// restores the state.
int autotune_mixed(mhd_bunch* b, int* chosen) {
    const int n = (int)b->cfg_index.size();
    std::vector<std::array<int, 3>> cls;
    std::vector<int> cls_of(b->npatch);
    for (int p = 0; p < b->npatch; ++p) {
        const std::array<int, 3> s = {b->pn[3 * p], b->pn[3 * p + 1], b->pn[3 * p + 2]};
        auto it = std::find(cls.begin(), cls.end(), s);
        cls_of[p] = (int)(it - cls.begin());
        if (it == cls.end()) cls.push_back(s);
    }
    std::vector<int> pick(cls.size(), 0);
    std::vector<int64_t> cells(cls.size(), 0);
    for (int p = 0; p < b->npatch; ++p) cells[cls_of[p]] += (int64_t)b->pn[3 * p] * b->pn[3 * p + 1] * b->pn[3 * p + 2];
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int4* d_tmp = nullptr;
    int rc = MHD_OK;
    cudaError_t e = cudaSuccess;
    for (size_t q = 0; q < cls.size() && rc == MHD_OK; ++q) {
        std::vector<char> sel(b->npatch);
        for (int p = 0; p < b->npatch; ++p) sel[p] = cls_of[p] == (int)q;
        float best = 1e30f;
        for (int c = 0; c < n && rc == MHD_OK; ++c) {
            const std::vector<int4> tl = class_tiles(b, c, sel);
            cudaFree(d_tmp);
            d_tmp = nullptr;
            e = cudaMalloc(&d_tmp, sizeof(int4) * tl.size());
            if (e == cudaSuccess)
                e = cudaMemcpy(d_tmp, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) break;
            const StepLaunch& L = step_cfg(b, c);
            int occ = 1;
            e = L.occupancy(&occ);
            if (e != cudaSuccess) break;
            StepHostArgs a = step_args(b, nullptr, 0.0);
            a.tiles = d_tmp;
            a.ntiles = (int)tl.size();
            a.dynamic = 1;
            const int grid = std::min((int)tl.size(), b->nsm * std::max(occ, 1));
            for (int w = 0; w < 6 && e == cudaSuccess; ++w) {
                if (w == 2) e = cudaEventRecord(e0, b->stream);
                if (e == cudaSuccess) e = L.launch(&a, grid, b->stream);
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) break;
            if (ms < best) {
                best = ms;
                pick[q] = c;
            }
        }
        if (e != cudaSuccess) rc = fail(MHD_ECUDA, cudaGetErrorString(e));
    }
    cudaFree(d_tmp);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    free_mixed(b);
    b->mixed.resize(n);
    for (int c = 0; c < n; ++c) {
        std::vector<char> sel(b->npatch);
        bool any = false;
        for (int p = 0; p < b->npatch; ++p) any |= (sel[p] = pick[cls_of[p]] == c) != 0;
        if (!any) continue;
        const std::vector<int4> tl = class_tiles(b, c, sel);
        CK(cudaMalloc(&b->mixed[c].d_tiles, sizeof(int4) * tl.size()));
        CK(cudaMemcpy(b->mixed[c].d_tiles, tl.data(), sizeof(int4) * tl.size(), cudaMemcpyHostToDevice));
        b->mixed[c].n = (int)tl.size();
    }
    if (chosen) *chosen = pick[std::max_element(cells.begin(), cells.end()) - cells.begin()];
    return MHD_OK;
}

// Step of the patches [p0, p1) only (U = current buffer -> the other one), one persistent
// launch over their tiles in natural order; the buffers are not swapped.
int do_step_range(mhd_bunch* b, const double* dt_ptr, int p0, int p1) {
    if (b->cfg_index.empty()) return fail(MHD_EINVAL, "no compiled kernel for this dimensionality");
    const int k = b->config < 0 ? default_config(b) : b->config;
    const StepLaunch& L = step_cfg(b, k);
    const auto& T = b->tiles[k];
    const int t0 = T.first[p0], t1 = p1 < b->npatch ? T.first[p1] : T.n;
    if (t1 <= t0) return MHD_OK;
    StepHostArgs a = step_args(b, dt_ptr, 0.0);
    int occ = 1;
    CK(L.occupancy(&occ));
    occ = std::max(occ, 1);
    a.tiles = T.d_nat + t0;
    a.ntiles = t1 - t0;
    a.dynamic = 1;
    CK(L.launch(&a, std::min(t1 - t0, b->nsm * occ), b->stream));
    b->launches++;
    return MHD_OK;
}

// Patch ranges of the streamed advances: at most K runs of contiguous patches.  When K
// equal runs would each hold at least one wave of the persistent update (SM count x
// occupancy tiles), the runs are cut at whole waves instead, so that no run's launch ends
// on a partly filled wave; smaller bunches are cut into K runs of about equal patch count.
int chunk_bounds(mhd_bunch* b, int K, std::vector<int>& pb) {
    const int P = b->npatch;
    K = std::max(1, std::min(K, P));
    pb.assign(1, 0);
    if (!b->cfg_index.empty()) {
        const int k = b->config < 0 ? default_config(b) : b->config;
        const auto& T = b->tiles[k];
        int occ = 1;
        CK(step_cfg(b, k).occupancy(&occ));
        const int64_t wave = (int64_t)b->nsm * std::max(occ, 1);
        const int64_t per = ((int64_t)T.n + K - 1) / K;
        if (wave > 0 && per >= wave) {
            const int64_t target = (per + wave - 1) / wave * wave;
            int64_t acc = 0;
            for (int p = 0; p + 1 < P; ++p) {
                acc += T.count[p];
                if (acc >= target) {
                    pb.push_back(p + 1);
                    acc = 0;
                }
            }
            pb.push_back(P);
            return MHD_OK;
        }
    }
    for (int c = 1; c <= K; ++c) pb.push_back((int)((int64_t)P * c / K));
    return MHD_OK;
}

int ensure_stream_pipeline(mhd_bunch* b, int nchunks) {
    if (!b->s_in) CK(cudaStreamCreateWithFlags(&b->s_in, cudaStreamNonBlocking));
    if (!b->s_out) CK(cudaStreamCreateWithFlags(&b->s_out, cudaStreamNonBlocking));
    while ((int)b->ev_in.size() < nchunks) {
        cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
        for (auto& x : e) CK(cudaEventCreateWithFlags(&x, cudaEventDisableTiming));
        b->ev_in.push_back(e[0]);
        b->ev_step.push_back(e[1]);
        b->ev_out.push_back(e[2]);
    }
    return MHD_OK;
}

// Neighbours of every patch for asynchronous stepping: the patches other than p that own a
// cell of p's guard zone (wrap / clamp as the guard fill).  Axes in the guard direction are
// walked cell by cell, the others by owner-map block.
void build_neighbours(mhd_bunch* b) {
    b->nbrs.assign(b->npatch, {});
    const int g = b->guard;
    for (int p = 0; p < b->npatch; ++p) {
        std::vector<int>& out = b->nbrs[p];
        for (int sz = -1; sz <= 1; ++sz)
            for (int sy = -1; sy <= 1; ++sy)
                for (int sx = -1; sx <= 1; ++sx) {
                    const int s3[3] = {sx, sy, sz};
                    if (!sx && !sy && !sz) continue;
                    int64_t lo[3], hi[3], st[3];
                    bool ok = true;
                    for (int d = 0; d < 3; ++d) {
                        const int64_t o = b->origin[3 * p + d], n = b->pn[3 * p + d];
                        if (n == 1 && s3[d] != 0) ok = false;
                        if (s3[d] < 0) { lo[d] = o - g; hi[d] = o; st[d] = 1; }
                        else if (s3[d] > 0) { lo[d] = o + n; hi[d] = o + n + g; st[d] = 1; }
                        else { lo[d] = o; hi[d] = o + n; st[d] = b->ob_bs[d]; }
                    }
                    if (!ok) continue;
                    for (int64_t z = lo[2]; z < hi[2]; z += st[2])
                        for (int64_t y = lo[1]; y < hi[1]; y += st[1])
                            for (int64_t x = lo[0]; x < hi[0]; x += st[0]) {
                                const int64_t c[3] = {x, y, z};
                                int64_t w[3];
                                for (int d = 0; d < 3; ++d) {
                                    const int64_t N = b->domain[d];
                                    if (c[d] < 0) w[d] = b->bc[2 * d] == MHD_BC_PERIODIC ? ((c[d] % N) + N) % N : 0;
                                    else if (c[d] >= N) w[d] = b->bc[2 * d + 1] == MHD_BC_PERIODIC ? c[d] % N : N - 1;
                                    else w[d] = c[d];
                                }
                                const int q = b->owner_h[(size_t)(((w[2] / b->ob_bs[2]) * b->ob_M[1] + w[1] / b->ob_bs[1]) *
                                                                  b->ob_M[0] + w[0] / b->ob_bs[0])];
                                if (q != p && std::find(out.begin(), out.end(), q) == out.end()) out.push_back(q);
                            }
                }
        std::sort(out.begin(), out.end());
    }
}

constexpr int kAsyncRows = 32;   // rounds enqueued between two reads of the record

int ensure_async(mhd_bunch* b) {
    if (b->nbrs.empty()) build_neighbours(b);
    const size_t P = (size_t)b->npatch;
    if (!b->d_slice) {
        std::vector<int> off(P + 1, 0), idx;
        for (size_t p = 0; p < P; ++p) {
            idx.insert(idx.end(), b->nbrs[p].begin(), b->nbrs[p].end());
            off[p + 1] = (int)idx.size();
        }
        CK(cudaMalloc(&b->d_slice, sizeof(int) * P));
        CK(cudaMalloc(&b->d_told, sizeof(double) * P));
        CK(cudaMalloc(&b->d_tcur, sizeof(double) * P));
        CK(cudaMalloc(&b->d_dtp, sizeof(double) * P));
        CK(cudaMalloc(&b->d_nb_off, sizeof(int) * (P + 1)));
        CK(cudaMalloc(&b->d_nb_idx, sizeof(int) * std::max<size_t>(idx.size(), 1)));
        CK(cudaMalloc(&b->d_tfirst, sizeof(int) * P));
        CK(cudaMalloc(&b->d_tcount, sizeof(int) * P));
        CK(cudaMalloc(&b->d_rows_list, sizeof(int) * P * kAsyncRows));
        CK(cudaMalloc(&b->d_rows_dt, sizeof(double) * P * kAsyncRows));
        CK(cudaMalloc(&b->d_rows_last, P * kAsyncRows));
        CK(cudaMalloc(&b->d_rows_n, sizeof(int) * kAsyncRows));
        CK(cudaMalloc(&b->d_ntiles, sizeof(int)));
        CK(cudaMalloc(&b->d_abort, sizeof(unsigned)));
        CK(cudaMalloc(&b->d_ready, sizeof(int) * P));
        CK(cudaMalloc(&b->d_rmax, sizeof(unsigned long long) * P));
        CK(cudaMemcpy(b->d_nb_off, off.data(), sizeof(int) * (P + 1), cudaMemcpyHostToDevice));
        if (!idx.empty()) CK(cudaMemcpy(b->d_nb_idx, idx.data(), sizeof(int) * idx.size(), cudaMemcpyHostToDevice));
    }
    return MHD_OK;
}

int read_error(mhd_bunch* b, int* code, char* msg, size_t len) {
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, b->stream));
    CK(cudaStreamSynchronize(b->stream));
    CK(cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), b->stream));
    int c = MHD_OK;
    std::string m;
    if (h & ERR_BOUNDS) {
        c = MHD_EBOUNDS;
        m = "device index outside the patch table";
    } else if (h & ERR_TIMEOUT) {
        c = MHD_ETIMEOUT;
        m = "a bounded device wait ran out";
    } else if (h & ERR_PHYS) {
        c = MHD_EPHYS;
        m = "non-physical state (rho <= 0 or non-finite value)";
    }
    if (code) *code = c;
    if (msg && len) {
        std::snprintf(msg, len, "%s", m.c_str());
    }
    if (c != MHD_OK) g_err = m;
    return MHD_OK;
}

}  // namespace

extern "C" {

int mhd_bunch_create(int nx, int ny, int nz, int guard, int nvar, int npatch, int real_bytes, mhd_bunch** out) try {
    if (npatch <= 0) return fail(MHD_EINVAL, "npatch must be positive");
    std::vector<int32_t> pn(3 * (size_t)npatch);
    for (int p = 0; p < npatch; ++p) {
        pn[3 * p] = nx;
        pn[3 * p + 1] = ny;
        pn[3 * p + 2] = nz;
    }
    return common_create(pn.data(), npatch, guard, nvar, real_bytes, out);
} MHD_CATCH_ALL

int mhd_bunch_create_ragged(const int32_t* patch_n, int npatch, int guard, int nvar, int real_bytes,
                            mhd_bunch** out) try {
    return common_create(patch_n, npatch, guard, nvar, real_bytes, out);
} MHD_CATCH_ALL

int mhd_bunch_set_geometry(mhd_bunch* b, const double dx[3], const int64_t* patch_origin,
                           const int64_t domain_cells[3], const int32_t bc[6]) try {
    if (!b || !dx || !patch_origin || !domain_cells || !bc) return fail(MHD_EINVAL, "NULL argument");
    if (b->slab) return fail(MHD_ESTATE, "the geometry of a slab handle is fixed");
    for (int d = 0; d < 3; ++d) {
        if (!(dx[d] > 0) || !std::isfinite(dx[d])) return fail(MHD_EINVAL, "dx must be positive");
        if (domain_cells[d] < 1 || domain_cells[d] > (1LL << 30)) return fail(MHD_EINVAL, "bad domain size");
        const bool act = domain_cells[d] > 1;
        if (act != (b->pn[d] > 1)) return fail(MHD_EINVAL, "collapsed axes of the box and the patches differ");
    }
    for (int k = 0; k < 6; ++k)
        if (bc[k] != MHD_BC_PERIODIC && bc[k] != MHD_BC_OUTFLOW) return fail(MHD_EINVAL, "bad boundary kind");
    // owner-map block = gcd of every patch size and origin and the box extent, per axis
    int64_t bs[3];
    for (int d = 0; d < 3; ++d) {
        int64_t g = domain_cells[d];
        for (int p = 0; p < b->npatch; ++p) {
            g = gcd64(g, b->pn[3 * p + d]);
            g = gcd64(g, patch_origin[3 * p + d]);
        }
        bs[d] = std::max<int64_t>(g, 1);
    }
    int64_t M[3];
    for (int d = 0; d < 3; ++d) M[d] = domain_cells[d] / bs[d];
    const int64_t ncell = M[0] * M[1] * M[2];
    if (ncell > (1LL << 28)) return fail(MHD_EINVAL, "owner map too large");
    std::vector<int> owner((size_t)ncell, -1);
    for (int p = 0; p < b->npatch; ++p) {
        int64_t lo[3], hi[3];
        for (int d = 0; d < 3; ++d) {
            lo[d] = patch_origin[3 * p + d];
            hi[d] = lo[d] + b->pn[3 * p + d];
            if (lo[d] < 0 || hi[d] > domain_cells[d]) return fail(MHD_EINVAL, "patch outside the box");
        }
        for (int64_t z = lo[2] / bs[2]; z < hi[2] / bs[2]; ++z)
            for (int64_t y = lo[1] / bs[1]; y < hi[1] / bs[1]; ++y)
                for (int64_t x = lo[0] / bs[0]; x < hi[0] / bs[0]; ++x) {
                    int& o = owner[(size_t)((z * M[1] + y) * M[0] + x)];
                    if (o != -1) return fail(MHD_EINVAL, "patches overlap");
                    o = p;
                }
    }
    for (int o : owner)
        if (o < 0) return fail(MHD_EINVAL, "patches do not cover the box");
    release_graph(b);
    b->owner_h = owner;
    for (int d = 0; d < 3; ++d) {
        b->ob_bs[d] = bs[d];
        b->ob_M[d] = M[d];
    }
    b->nbrs.clear();
    cudaFree(b->d_owner);
    b->d_owner = nullptr;
    CK(cudaMalloc(&b->d_owner, sizeof(int) * owner.size()));
    CK(cudaMemcpy(b->d_owner, owner.data(), sizeof(int) * owner.size(), cudaMemcpyHostToDevice));
    for (int d = 0; d < 3; ++d) {
        b->dx[d] = dx[d];
        b->domain[d] = domain_cells[d];
        b->fg.N[d] = (int)domain_cells[d];
        b->fg.bs[d] = (int)bs[d];
        b->fg.M[d] = (int)M[d];
        b->fg.bc[d][0] = bc[2 * d];
        b->fg.bc[d][1] = bc[2 * d + 1];
    }
    for (int k = 0; k < 6; ++k) b->bc[k] = bc[k];
    b->fg.owner = b->d_owner;
    b->origin.assign(patch_origin, patch_origin + 3 * b->npatch);
    for (int p = 0; p < b->npatch; ++p) {
        b->hp[p].ox = (int)patch_origin[3 * p];
        b->hp[p].oy = (int)patch_origin[3 * p + 1];
        b->hp[p].oz = (int)patch_origin[3 * p + 2];
        // the patch's sides that are outflow box faces (zero-gradient ghosts)
        int cl = 0;
        for (int d = 0; d < 3; ++d) {
            if (b->pn[3 * p + d] == 1) continue;
            if (bc[2 * d] == MHD_BC_OUTFLOW && patch_origin[3 * p + d] == 0) cl |= 1 << (2 * d);
            if (bc[2 * d + 1] == MHD_BC_OUTFLOW && patch_origin[3 * p + d] + b->pn[3 * p + d] == domain_cells[d])
                cl |= 2 << (2 * d);
        }
        b->hp[p].clamp = cl;
    }
    {
        const std::vector<int64_t> t = neighbour_table(b, patch_origin, domain_cells, owner, bs, M);
        cudaFree(b->d_nboff);
        b->d_nboff = nullptr;
        cudaFree(b->d_partial_fc);
        b->d_partial_fc = nullptr;
        if (!t.empty()) {
            CK(cudaMalloc(&b->d_partial_fc, (size_t)b->npatch * b->hp[0].Z * b->rb));
            CK(cudaMalloc(&b->d_nboff, sizeof(int64_t) * t.size()));
            CK(cudaMemcpy(b->d_nboff, t.data(), sizeof(int64_t) * t.size(), cudaMemcpyHostToDevice));
        }
    }
    CK(cudaMemcpy(b->d_patches, b->hp.data(), sizeof(PatchDev) * b->npatch, cudaMemcpyHostToDevice));
    int rc = build_tiles(b);
    if (rc != MHD_OK) return rc;
    b->have_geom = true;
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_set_slab(mhd_bunch* b, int z0, int z1) try {
    if (!b) return fail(MHD_EINVAL, "handle is NULL");
    if (!b->have_geom) return fail(MHD_ESTATE, "mhd_bunch_set_geometry has not been called");
    if (b->slab) return fail(MHD_ESTATE, "the handle is a slab already");
    if (b->ndim != 3) return fail(MHD_EINVAL, "slabs need a 3D box");
    const int P = b->npatch;
    const int nx = b->pn[0], ny = b->pn[1], nz = b->pn[2];
    int64_t np3[3];
    for (int d = 0; d < 3; ++d) np3[d] = b->domain[d] / b->pn[d];
    const int64_t ppl = np3[0] * np3[1];
    const int NL = (int)np3[2];
    bool grid = ppl * NL == P && b->d_nboff != nullptr;
    for (int p = 0; p < P && grid; ++p)
        grid = b->pn[3 * p] == nx && b->pn[3 * p + 1] == ny && b->pn[3 * p + 2] == nz &&
               b->origin[3 * p] == (p % np3[0]) * nx && b->origin[3 * p + 1] == ((p / np3[0]) % np3[1]) * ny &&
               b->origin[3 * p + 2] == (p / ppl) * nz;
    if (!grid) return fail(MHD_EINVAL, "slabs need equal patches on a grid, x fastest in patch order");
    if (ppl > 65535) return fail(MHD_EINVAL, "more than 65535 patches per z-layer");
    if (z0 < 0 || z1 > NL || z0 >= z1) return fail(MHD_EINVAL, "need 0 <= z0 < z1 <= number of patch layers");
    const int L = z1 - z0;
    const PatchDev h0 = b->hp[0];
    const int64_t pe = 8LL * h0.X * h0.Y * h0.Z;
    const bool per_lo = b->bc[4] == MHD_BC_PERIODIC, per_hi = b->bc[5] == MHD_BC_PERIODIC;
    // slot of layer g (z-neighbour direction sz) as seen from an owned layer
    auto slot_of = [&](int g, int sz, int gown) -> int {
        if (g < 0 || g >= NL) {
            if ((g < 0 && !per_lo) || (g >= NL && !per_hi)) return gown - z0;   // outflow: never read
            g = (g + NL) % NL;
        }
        if (g >= z0 && g < z1) return g - z0;
        return sz < 0 ? L : L + 1;
    };
    std::vector<PatchDev> hp;
    std::vector<int64_t> offs, nb;
    std::vector<int> pn;
    std::vector<int64_t> origin;
    for (int g = z0; g < z1; ++g)
        for (int64_t j = 0; j < ppl; ++j) {
            const int p = (int)(g * ppl + j);
            PatchDev q = b->hp[p];
            q.off = ((int64_t)(g - z0) * ppl + j) * pe;
            hp.push_back(q);
            offs.push_back(q.off);
            for (int d = 0; d < 3; ++d) {
                pn.push_back(b->pn[3 * p + d]);
                origin.push_back(b->origin[3 * p + d]);
            }
            const int64_t ix = j % np3[0], iy = j / np3[0];
            for (int sz = -1; sz <= 1; ++sz)
                for (int sy = -1; sy <= 1; ++sy)
                    for (int sx = -1; sx <= 1; ++sx) {
                        const int64_t jx = ((ix + sx) % np3[0] + np3[0]) % np3[0];
                        const int64_t jy = ((iy + sy) % np3[1] + np3[1]) % np3[1];
                        nb.push_back(((int64_t)slot_of(g + sz, sz, g) * ppl + jy * np3[0] + jx) * pe);
                    }
        }
    std::vector<PatchDev> slots((size_t)(L + 2) * ppl);
    for (int sl = 0; sl < L + 2; ++sl)
        for (int64_t j = 0; j < ppl; ++j) {
            PatchDev q = h0;
            q.off = ((int64_t)sl * ppl + j) * pe;
            slots[(size_t)sl * ppl + j] = q;
        }
    std::vector<int64_t> ioff(ppl);
    for (int64_t j = 0; j < ppl; ++j) ioff[j] = j * 8LL * nx * ny * nz;
    release_graph(b);
    free_tiles(b);
    cudaFree(b->d_patches);
    b->d_patches = nullptr;
    cudaFree(b->d_nboff);
    b->d_nboff = nullptr;
    cudaFree(b->d_partial_fc);
    b->d_partial_fc = nullptr;
    b->npatch = L * (int)ppl;
    b->hp = hp;
    b->offs = offs;
    b->pn = pn;
    b->origin = origin;
    b->state_bytes = (size_t)(L + 2) * ppl * pe * b->rb;
    b->buf[0] = b->buf[1] = nullptr;       // bind buffers of the slab's size
    b->ioff_h.clear();
    CK(cudaMalloc(&b->d_patches, sizeof(PatchDev) * hp.size()));
    CK(cudaMemcpy(b->d_patches, hp.data(), sizeof(PatchDev) * hp.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&b->d_nboff, sizeof(int64_t) * nb.size()));
    CK(cudaMemcpy(b->d_nboff, nb.data(), sizeof(int64_t) * nb.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&b->d_partial_fc, (size_t)b->npatch * h0.Z * b->rb));
    CK(cudaMalloc(&b->d_slab_slots, sizeof(PatchDev) * slots.size()));
    CK(cudaMemcpy(b->d_slab_slots, slots.data(), sizeof(PatchDev) * slots.size(), cudaMemcpyHostToDevice));
    CK(cudaMalloc(&b->d_slab_ioff, sizeof(int64_t) * ppl));
    CK(cudaMemcpy(b->d_slab_ioff, ioff.data(), sizeof(int64_t) * ppl, cudaMemcpyHostToDevice));
    b->slab = true;
    b->slab_z0 = z0;
    b->slab_z1 = z1;
    b->slab_nl = NL;
    b->slab_ppl = ppl;
    return build_tiles(b);
} MHD_CATCH_ALL

int mhd_bunch_slab_info(const mhd_bunch* b, int* layers, int64_t* patches_per_layer, size_t* layer_bytes) try {
    if (!b || !layers || !patches_per_layer || !layer_bytes) return fail(MHD_EINVAL, "NULL argument");
    if (!b->slab) return fail(MHD_ESTATE, "not a slab handle");
    *layers = b->slab_z1 - b->slab_z0;
    *patches_per_layer = b->slab_ppl;
    *layer_bytes = (size_t)b->slab_ppl * 8 * b->pn[0] * b->pn[1] * b->pn[2] * b->rb;
    return MHD_OK;
} MHD_CATCH_ALL

// interior of layer slot sl of the current state <-> a buffer in the interior layout
int slab_copy(mhd_bunch* b, int sl, void* buf, int to_padded) {
    const int nz = b->pn[2];
    interior_copy_kernel<<<dim3(nz, (unsigned)b->slab_ppl), 256, 0, b->stream>>>(
        static_cast<unsigned*>(b->buf[b->cur]), static_cast<unsigned*>(buf), b->d_slab_slots + (size_t)sl * b->slab_ppl,
        b->d_slab_ioff, 0, (int)b->slab_ppl, b->rb / 4, to_padded);
    ++b->launches;
    CK(cudaGetLastError());
    return MHD_OK;
}

int mhd_bunch_slab_pack(mhd_bunch* b, void* bottom, void* top) try {
    int rc = ready(b);
    if (rc) return rc;
    if (!b->slab) return fail(MHD_ESTATE, "not a slab handle");
    if (bottom && (rc = slab_copy(b, 0, bottom, 0))) return rc;
    if (top && (rc = slab_copy(b, b->slab_z1 - b->slab_z0 - 1, top, 0))) return rc;
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_slab_unpack(mhd_bunch* b, const void* below, const void* above) try {
    int rc = ready(b);
    if (rc) return rc;
    if (!b->slab) return fail(MHD_ESTATE, "not a slab handle");
    const int L = b->slab_z1 - b->slab_z0;
    if (below && (rc = slab_copy(b, L, const_cast<void*>(below), 1))) return rc;
    if (above && (rc = slab_copy(b, L + 1, const_cast<void*>(above), 1))) return rc;
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_set_params(mhd_bunch* b, double gamma, double courant, int limiter) try {
    if (!b) return fail(MHD_EINVAL, "handle is NULL");
    if (!(gamma > 1.0) || !std::isfinite(gamma)) return fail(MHD_EINVAL, "gamma must be > 1");
    if (!(courant > 0.0) || !std::isfinite(courant)) return fail(MHD_EINVAL, "courant must be > 0");
    if (limiter != MHD_LIMITER_MINMOD && limiter != MHD_LIMITER_MC) return fail(MHD_EINVAL, "bad limiter");
    release_graph(b);
    b->gamma = gamma;
    b->courant = courant;
    b->limiter = limiter;
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_set_riemann(mhd_bunch* b, int solver) try {
    if (!b) return fail(MHD_EINVAL, "handle is NULL");
    if (solver != MHD_RIEMANN_HLLD && solver != MHD_RIEMANN_HLL) return fail(MHD_EINVAL, "bad face-flux solver");
    release_graph(b);
    b->riemann = solver;
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_set_bunches(mhd_bunch* b, const int32_t* patches, const int32_t* starts, int nbunch) try {
    if (!b || !patches || !starts) return fail(MHD_EINVAL, "NULL argument");
    if (!b->have_geom) return fail(MHD_ESTATE, "set_geometry first");
    if (nbunch < 1 || nbunch > b->npatch) return fail(MHD_EINVAL, "nbunch must be in 1..npatch");
    if (starts[0] != 0 || starts[nbunch] != b->npatch)
        return fail(MHD_EINVAL, "starts must run from 0 to npatch");
    std::vector<char> seen(b->npatch, 0);
    for (int q = 0; q < nbunch; ++q) {
        if (starts[q + 1] <= starts[q]) return fail(MHD_EINVAL, "every bunch must hold at least one patch");
        for (int i = starts[q]; i < starts[q + 1]; ++i) {
            const int p = patches[i];
            if (p < 0 || p >= b->npatch || seen[p]) return fail(MHD_EINVAL, "patches must list every patch once");
            seen[p] = 1;
        }
    }
    release_graph(b);
    free_btiles(b);
    b->bunch_patches.assign(patches, patches + b->npatch);
    b->bunch_start.assign(starts, starts + nbunch + 1);
    b->btiles.resize(b->tiles.size());
    for (size_t k = 0; k < b->tiles.size(); ++k) {
        const auto& T = b->tiles[k];
        auto& BT = b->btiles[k];
        std::vector<int4> all;
        for (int q = 0; q < nbunch; ++q) {
            std::vector<int4> tl;
            for (int i = starts[q]; i < starts[q + 1]; ++i) {
                const int p = patches[i];
                tl.insert(tl.end(), T.nat_h.begin() + T.first[p], T.nat_h.begin() + T.first[p] + T.count[p]);
            }
            std::stable_sort(tl.begin(), tl.end(), [](const int4& x, const int4& y) { return x.w > y.w; });
            BT.first.push_back((int)all.size());
            BT.count.push_back((int)tl.size());
            all.insert(all.end(), tl.begin(), tl.end());
        }
        CK(cudaMalloc(&BT.d_tiles, sizeof(int4) * all.size()));
        CK(cudaMemcpy(BT.d_tiles, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice));
    }
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_interior_size(const mhd_bunch* b, size_t* bytes, int64_t* patch_offsets) try {
    if (!b || !bytes) return fail(MHD_EINVAL, "NULL argument");
    int64_t o = 0;
    for (int p = 0; p < b->npatch; ++p) {
        if (patch_offsets) patch_offsets[p] = o;
        o += 8 * (int64_t)b->pn[3 * p] * b->pn[3 * p + 1] * b->pn[3 * p + 2];
    }
    *bytes = (size_t)o * b->rb;
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_state_size(const mhd_bunch* b, size_t* bytes, int64_t* patch_offsets) try {
    if (!b || !bytes) return fail(MHD_EINVAL, "NULL argument");
    *bytes = b->state_bytes;
    if (patch_offsets) std::copy(b->offs.begin(), b->offs.end(), patch_offsets);
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_bind(mhd_bunch* b, void* state, void* state_next, void* cuda_stream) try {
    if (!b || !state || !state_next) return fail(MHD_EINVAL, "NULL argument");
    if (state == state_next) return fail(MHD_EINVAL, "state and state_next must differ");
    if ((reinterpret_cast<uintptr_t>(state) & 15) || (reinterpret_cast<uintptr_t>(state_next) & 15))
        return fail(MHD_EINVAL, "state buffers must be 16-byte aligned");
    release_graph(b);
    b->buf[0] = state;
    b->buf[1] = state_next;
    b->cur = 0;
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_current(const mhd_bunch* b, void** state) try {
    if (!b || !state) return fail(MHD_EINVAL, "NULL argument");
    *state = b->buf[b->cur];
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_fill_guards(mhd_bunch* b) try {
    int rc = ready(b);
    if (rc) return rc;
    return do_fill(b);
} MHD_CATCH_ALL

int mhd_bunch_cfl_dt_device(mhd_bunch* b, void* dt_dev) try {
    int rc = ready(b);
    if (rc) return rc;
    if (!dt_dev) return fail(MHD_EINVAL, "dt_dev is NULL");
    return do_cfl(b, static_cast<double*>(dt_dev));
} MHD_CATCH_ALL

int mhd_bunch_fill_cfl_device(mhd_bunch* b, void* dt_dev) try {
    int rc = ready(b);
    if (rc) return rc;
    if (!dt_dev) return fail(MHD_EINVAL, "dt_dev is NULL");
    return do_fill_cfl(b, static_cast<double*>(dt_dev));
} MHD_CATCH_ALL

int mhd_bunch_cfl_dt(mhd_bunch* b, double* dt_host) try {
    int rc = ready(b);
    if (rc) return rc;
    if (!dt_host) return fail(MHD_EINVAL, "dt_host is NULL");
    rc = do_cfl(b, b->d_dt);
    if (rc) return rc;
    CK(cudaMemcpyAsync(dt_host, b->d_dt, sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    int code = 0;
    rc = read_error(b, &code, nullptr, 0);
    if (rc) return rc;
    return code;
} MHD_CATCH_ALL

int mhd_bunch_step(mhd_bunch* b, double dt) try {
    int rc = ready(b);
    if (rc) return rc;
    if (!(dt >= 0) || !std::isfinite(dt)) return fail(MHD_EINVAL, "dt must be finite and >= 0");
    return do_step(b, nullptr, dt);
} MHD_CATCH_ALL

int mhd_bunch_step_device_dt(mhd_bunch* b, const void* dt_dev) try {
    int rc = ready(b);
    if (rc) return rc;
    if (!dt_dev) return fail(MHD_EINVAL, "dt_dev is NULL");
    return do_step(b, static_cast<const double*>(dt_dev), 0.0);
} MHD_CATCH_ALL

int mhd_bunch_set_mode(mhd_bunch* b, int mode, int config) try {
    if (!b) return fail(MHD_EINVAL, "handle is NULL");
    if (mode < MHD_MODE_PER_PATCH || mode > MHD_MODE_BUNCH_LISTS) return fail(MHD_EINVAL, "bad mode");
    if (config < -1 || config >= (int)b->cfg_index.size()) return fail(MHD_EINVAL, "bad config index");
    release_graph(b);
    b->mode = mode;
    b->config = config;
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_num_configs(const mhd_bunch* b, int* nconfig) try {
    if (!b || !nconfig) return fail(MHD_EINVAL, "NULL argument");
    *nconfig = (int)b->cfg_index.size();
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_config_info(const mhd_bunch* b, int config, int* tile_x, int* tile_y, int* threads) try {
    if (!b) return fail(MHD_EINVAL, "handle is NULL");
    if (config < 0 || config >= (int)b->cfg_index.size()) return fail(MHD_EINVAL, "bad config index");
    const StepLaunch& L = step_cfg(b, config);
    if (tile_x) *tile_x = L.tx;
    if (tile_y) *tile_y = L.ty;
    if (threads) *threads = L.nt;
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_autotune(mhd_bunch* b, const char* cache_path, int* chosen) try {
    int rc = ready(b);
    if (rc) return rc;
    const int n = (int)b->cfg_index.size();
    if (n == 0) return fail(MHD_EINVAL, "no compiled kernel for this dimensionality");
    // cache key: device name, precision, dimensionality and the multiset of patch sizes
    cudaDeviceProp prop;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaGetDeviceProperties(&prop, dev));
    std::ostringstream key;
    key << prop.name << "|r" << b->rb << "|d" << b->ndim << "|m" << b->mode;
    {
        std::vector<int> sizes;
        for (int p = 0; p < b->npatch; ++p) sizes.push_back(b->pn[3 * p] * 10000 + b->pn[3 * p + 1] * 100 + b->pn[3 * p + 2]);
        std::sort(sizes.begin(), sizes.end());
        int64_t h = 1469598103934665603LL;
        for (int s : sizes) h = (h ^ s) * 1099511628211LL;
        key << "|p" << b->npatch << "|h" << (uint64_t)h;
    }
    std::string k = key.str();
    for (auto& ch : k)
        if (ch == ' ') ch = '_';
    if (cache_path && b->mode != MHD_MODE_MIXED) {
        std::ifstream f(cache_path);
        std::string kk;
        int idx;
        while (f >> kk >> idx)
            if (kk == k && idx >= 0 && idx < n) {
                release_graph(b);
                b->config = idx;
                if (chosen) *chosen = idx;
                return MHD_OK;
            }
    }
    // time every configuration on the bound state, then restore it
    void* save = nullptr;
    CK(cudaMalloc(&save, b->state_bytes));
    const int cur0 = b->cur;
    cudaError_t e = cudaMemcpyAsync(save, b->buf[cur0], b->state_bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e != cudaSuccess) {
        cudaFree(save);
        return fail(MHD_ECUDA, cudaGetErrorString(e));
    }
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int keep = b->config;
    float best = 1e30f;
    int besti = 0;
    rc = do_fill(b);
    const bool mixed = b->mode == MHD_MODE_MIXED;
    if (mixed && rc == MHD_OK) rc = autotune_mixed(b, &besti);
    for (int c = 0; c < n && rc == MHD_OK && !mixed; ++c) {
        b->config = c;
        // dt = 0 keeps the state unchanged in value; the work is the same as a real step
        for (int w = 0; w < 2 && rc == MHD_OK; ++w) {
            rc = do_fill(b);
            if (!rc) rc = do_step(b, nullptr, 0.0);
        }
        if (rc) break;
        e = cudaEventRecord(e0, b->stream);
        for (int w = 0; w < 4 && rc == MHD_OK; ++w) {
            rc = do_fill(b);
            if (!rc) rc = do_step(b, nullptr, 0.0);
        }
        if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
            rc = fail(MHD_ECUDA, cudaGetErrorString(e));
            break;
        }
        if (ms < best) {
            best = ms;
            besti = c;
        }
    }
    // restore the state into the buffer that held it
    b->cur = cur0;
    e = cudaMemcpyAsync(b->buf[cur0], save, b->state_bytes, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    cudaFree(save);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) {
        b->config = keep;
        return rc;
    }
    if (e != cudaSuccess) return fail(MHD_ECUDA, cudaGetErrorString(e));
    release_graph(b);
    if (!mixed) b->config = besti;
    if (chosen) *chosen = besti;
    if (cache_path && !mixed) {
        std::ofstream f(cache_path, std::ios::app);
        f << k << " " << besti << "\n";
    }
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_graph_capture(mhd_bunch* b, int nsteps, void* dt_dev) try {
    int rc = ready(b);
    if (rc) return rc;
    if (nsteps <= 0) return fail(MHD_EINVAL, "nsteps must be positive");
    release_graph(b);
    const int cur0 = b->cur;
    const int64_t l0 = b->launches;
    // an even sequence returns to its starting buffer: one graph; an odd one swaps, so a
    // second graph starting from the other buffer is captured as well
    const int ngraphs = (nsteps & 1) ? 2 : 1;
    for (int gi = 0; gi < ngraphs; ++gi) {
        b->cur = gi == 0 ? cur0 : 1 - cur0;
        CK(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
        for (int s = 0; s < nsteps && rc == MHD_OK; ++s) {
            double* dt = dt_dev ? static_cast<double*>(dt_dev) + s : b->d_dt;
            rc = do_fill_cfl(b, dt);
            if (!rc) rc = do_step(b, dt, 0.0);
        }
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->stream, &g);
        if (rc || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            b->cur = cur0;
            b->launches = l0;
            release_graph(b);
            return rc ? rc : fail(MHD_ECUDA, std::string("capture: ") + cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&b->gexec[gi], g, 0);
        b->graph[gi] = g;
        if (e != cudaSuccess) {
            b->cur = cur0;
            b->launches = l0;
            release_graph(b);
            return fail(MHD_ECUDA, std::string("instantiate: ") + cudaGetErrorString(e));
        }
    }
    b->cur = cur0;
    b->launches = l0;
    b->graph_steps = nsteps;
    b->graph_start = cur0;
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_graph_launch(mhd_bunch* b) try {
    int rc = ready(b);
    if (rc) return rc;
    if (!b->gexec[0]) return fail(MHD_ESTATE, "no captured graph");
    const int gi = (b->cur == b->graph_start) ? 0 : 1;
    if (!b->gexec[gi]) return fail(MHD_ESTATE, "current buffer differs from the captured one");
    CK(cudaGraphLaunch(b->gexec[gi], b->stream));
    size_t nn = 0;
    cudaGraphGetNodes(b->graph[gi], nullptr, &nn);
    b->launches += (int64_t)nn;
    if (b->graph_steps & 1) b->cur = 1 - b->cur;
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_advance_host(mhd_bunch* b, void* host_state, int nsteps, double* t_out) try {
    if (b && b->slab) return not_slab(b);
    int rc = ready(b);
    if (rc) return rc;
    if (!host_state || nsteps < 0) return fail(MHD_EINVAL, "bad argument");
    if (nsteps > b->d_dts_cap) {
        cudaFree(b->d_dts);
        b->d_dts = nullptr;
        CK(cudaMalloc(&b->d_dts, sizeof(double) * nsteps));
        b->d_dts_cap = nsteps;
    }
    CK(cudaMemcpyAsync(b->buf[b->cur], host_state, b->state_bytes, cudaMemcpyHostToDevice, b->stream));
    for (int s = 0; s < nsteps; ++s) {
        rc = do_fill_cfl(b, b->d_dts + s);
        if (!rc) rc = do_step(b, b->d_dts + s, 0.0);
        if (rc) return rc;
    }
    std::vector<double> dts(nsteps);
    if (nsteps) CK(cudaMemcpyAsync(dts.data(), b->d_dts, sizeof(double) * nsteps, cudaMemcpyDeviceToHost, b->stream));
    CK(cudaMemcpyAsync(host_state, b->buf[b->cur], b->state_bytes, cudaMemcpyDeviceToHost, b->stream));
    int code = 0;
    rc = read_error(b, &code, nullptr, 0);
    if (rc) return rc;
    if (t_out) *t_out = std::accumulate(dts.begin(), dts.end(), 0.0);
    return code;
} MHD_CATCH_ALL

int mhd_bunch_advance_streamed(mhd_bunch* b, void* host_state, int nsteps, int nchunks, double* t_out) try {
    if (b && b->slab) return not_slab(b);
    int rc = ready(b);
    if (rc) return rc;
    if (!host_state || nsteps < 1 || nchunks < 1) return fail(MHD_EINVAL, "bad argument");
    if (b->stream == nullptr) return fail(MHD_EINVAL, "the bound stream must not be the legacy default stream");
    if (nsteps > b->d_dts_cap) {
        cudaFree(b->d_dts);
        b->d_dts = nullptr;
        CK(cudaMalloc(&b->d_dts, sizeof(double) * nsteps));
        b->d_dts_cap = nsteps;
    }
    // chunks: contiguous patch ranges (chunk_bounds); bytes [bo[k], bo[k+1])
    std::vector<int> pb;
    rc = chunk_bounds(b, nchunks, pb);
    if (rc) return rc;
    const int K = (int)pb.size() - 1;
    rc = ensure_stream_pipeline(b, K);
    if (rc) return rc;
    std::vector<size_t> bo(K + 1);
    for (int k = 0; k <= K; ++k) bo[k] = pb[k] < b->npatch ? (size_t)b->offs[pb[k]] * b->rb : b->state_bytes;
    char* host = static_cast<char*>(host_state);
    const int A = b->cur, B = 1 - A;
    char* dA = static_cast<char*>(b->buf[A]);
    char* dB = static_cast<char*>(b->buf[B]);
    // the copy streams start after the work already queued on the bound stream
    CK(cudaEventRecord(b->ev_step[0], b->stream));
    CK(cudaStreamWaitEvent(b->s_in, b->ev_step[0], 0));
    CK(cudaStreamWaitEvent(b->s_out, b->ev_step[0], 0));
    for (int s = 0; s < nsteps; ++s) {
        // upload: chunk k of the host state, once the previous step's chunk k is back
        for (int k = 0; k < K; ++k) {
            if (s > 0) CK(cudaStreamWaitEvent(b->s_in, b->ev_out[k], 0));
            CK(cudaMemcpyAsync(dA + bo[k], host + bo[k], bo[k + 1] - bo[k], cudaMemcpyHostToDevice, b->s_in));
            CK(cudaEventRecord(b->ev_in[k], b->s_in));
        }
        for (int k = 0; k < K; ++k) CK(cudaStreamWaitEvent(b->stream, b->ev_in[k], 0));
        // guard fill and dt need the whole state; the update runs chunk by chunk and each
        // chunk goes back to the host as soon as it is done
        b->cur = A;
        rc = do_fill_cfl(b, b->d_dts + s);
        for (int k = 0; k < K && !rc; ++k) {
            rc = do_step_range(b, b->d_dts + s, pb[k], pb[k + 1]);
            if (rc) break;
            CK(cudaEventRecord(b->ev_step[k], b->stream));
            CK(cudaStreamWaitEvent(b->s_out, b->ev_step[k], 0));
            CK(cudaMemcpyAsync(host + bo[k], dB + bo[k], bo[k + 1] - bo[k], cudaMemcpyDeviceToHost, b->s_out));
            CK(cudaEventRecord(b->ev_out[k], b->s_out));
        }
        if (rc) {
            b->cur = A;
            cudaStreamSynchronize(b->s_in);
            cudaStreamSynchronize(b->s_out);
            return rc;
        }
    }
    // join: the bound stream waits for the last downloads; B holds the final state
    for (int k = 0; k < K; ++k) CK(cudaStreamWaitEvent(b->stream, b->ev_out[k], 0));
    b->cur = B;
    std::vector<double> dts(nsteps);
    CK(cudaMemcpyAsync(dts.data(), b->d_dts, sizeof(double) * nsteps, cudaMemcpyDeviceToHost, b->stream));
    int code = 0;
    rc = read_error(b, &code, nullptr, 0);
    if (rc) return rc;
    if (t_out) *t_out = std::accumulate(dts.begin(), dts.end(), 0.0);
    return code;
} MHD_CATCH_ALL

int mhd_bunch_advance_streamed_interior(mhd_bunch* b, void* host_interior, int nsteps, int nchunks,
                                        double* t_out) try {
    if (b && b->slab) return not_slab(b);
    int rc = ready(b);
    if (rc) return rc;
    if (!host_interior || nsteps < 1 || nchunks < 1) return fail(MHD_EINVAL, "bad argument");
    if (b->stream == nullptr) return fail(MHD_EINVAL, "the bound stream must not be the legacy default stream");
    const int P = b->npatch;
    if (nsteps > b->d_dts_cap) {
        cudaFree(b->d_dts);
        b->d_dts = nullptr;
        CK(cudaMalloc(&b->d_dts, sizeof(double) * nsteps));
        b->d_dts_cap = nsteps;
    }
    for (const auto& q : b->hp)   // the copy kernel indexes within a patch in 32 bits
        if ((int64_t)8 * q.X * q.Y * q.Z * (b->rb / 4) >= ((int64_t)1 << 31))
            return fail(MHD_EINVAL, "a patch is too large for the interior-layout stream (2^31 words)");
    std::vector<int> pb;
    rc = chunk_bounds(b, nchunks, pb);
    if (rc) return rc;
    const int K = (int)pb.size() - 1;
    rc = ensure_stream_pipeline(b, K);
    if (rc) return rc;
    size_t ibytes = 0;
    if (b->ioff_h.empty()) {
        std::vector<int64_t> io(P);
        mhd_bunch_interior_size(b, &ibytes, io.data());
        CK(cudaMalloc(&b->d_ioff, sizeof(int64_t) * P));
        CK(cudaMemcpy(b->d_ioff, io.data(), sizeof(int64_t) * P, cudaMemcpyHostToDevice));
        CK(cudaMalloc(&b->d_interior, ibytes));
        b->ioff_h = std::move(io);
    }
    mhd_bunch_interior_size(b, &ibytes, nullptr);
    // chunks (chunk_bounds); interior bytes [bo[k], bo[k+1])
    std::vector<size_t> bo(K + 1);
    int maxnz = 1;
    for (int p = 0; p < P; ++p) maxnz = std::max(maxnz, (int)b->pn[3 * p + 2]);
    for (int k = 0; k <= K; ++k) bo[k] = pb[k] < P ? (size_t)b->ioff_h[pb[k]] * b->rb : ibytes;
    char* host = static_cast<char*>(host_interior);
    char* stage = static_cast<char*>(b->d_interior);
    const int A = b->cur, B = 1 - A;
    const int wpr = b->rb / 4;
    auto copy = [&](int k, int buf, int to_padded) -> cudaError_t {
        const dim3 grid(maxnz, pb[k + 1] - pb[k]);
        interior_copy_kernel<<<grid, 256, 0, b->stream>>>(static_cast<unsigned*>(b->buf[buf]),
                                                          static_cast<unsigned*>(b->d_interior), b->d_patches, b->d_ioff,
                                                          pb[k], pb[k + 1], wpr, to_padded);
        ++b->launches;
        return cudaGetLastError();
    };
    // the copy streams start after the work already queued on the bound stream
    CK(cudaEventRecord(b->ev_step[0], b->stream));
    CK(cudaStreamWaitEvent(b->s_in, b->ev_step[0], 0));
    CK(cudaStreamWaitEvent(b->s_out, b->ev_step[0], 0));
    for (int s = 0; s < nsteps; ++s) {
        // upload chunk k into the staging buffer once the previous step's chunk k is back on
        // the host (its staging bytes are free then too), and scatter it into the state
        for (int k = 0; k < K; ++k) {
            if (s > 0) CK(cudaStreamWaitEvent(b->s_in, b->ev_out[k], 0));
            CK(cudaMemcpyAsync(stage + bo[k], host + bo[k], bo[k + 1] - bo[k], cudaMemcpyHostToDevice, b->s_in));
            CK(cudaEventRecord(b->ev_in[k], b->s_in));
        }
        for (int k = 0; k < K; ++k) {
            CK(cudaStreamWaitEvent(b->stream, b->ev_in[k], 0));
            CK(copy(k, A, 1));
        }
        // guard fill and dt need the whole state; the update runs chunk by chunk, each
        // updated chunk gathered into the staging buffer and sent back to the host
        b->cur = A;
        rc = do_fill_cfl(b, b->d_dts + s);
        for (int k = 0; k < K && !rc; ++k) {
            rc = do_step_range(b, b->d_dts + s, pb[k], pb[k + 1]);
            if (rc) break;
            CK(copy(k, B, 0));
            CK(cudaEventRecord(b->ev_step[k], b->stream));
            CK(cudaStreamWaitEvent(b->s_out, b->ev_step[k], 0));
            CK(cudaMemcpyAsync(host + bo[k], stage + bo[k], bo[k + 1] - bo[k], cudaMemcpyDeviceToHost, b->s_out));
            CK(cudaEventRecord(b->ev_out[k], b->s_out));
        }
        if (rc) {
            b->cur = A;
            cudaStreamSynchronize(b->s_in);
            cudaStreamSynchronize(b->s_out);
            return rc;
        }
    }
    // join: the bound stream waits for the last downloads; B holds the final state
    for (int k = 0; k < K; ++k) CK(cudaStreamWaitEvent(b->stream, b->ev_out[k], 0));
    b->cur = B;
    std::vector<double> dts(nsteps);
    CK(cudaMemcpyAsync(dts.data(), b->d_dts, sizeof(double) * nsteps, cudaMemcpyDeviceToHost, b->stream));
    int code = 0;
    rc = read_error(b, &code, nullptr, 0);
    if (rc) return rc;
    if (t_out) *t_out = std::accumulate(dts.begin(), dts.end(), 0.0);
    return code;
} MHD_CATCH_ALL

int mhd_bunch_advance_out_of_core(mhd_bunch* b, void* host_state, void* host_scratch, int nsteps,
                                  size_t device_budget, void* cuda_stream, double* t_out, size_t* io_bytes) try {
    if (!b) return fail(MHD_EINVAL, "handle is NULL");
    if (!b->have_geom) return fail(MHD_ESTATE, "mhd_bunch_set_geometry has not been called");
    if (b->slab) return not_slab(b);
    if (!host_state || !host_scratch || host_state == host_scratch || nsteps < 1 || device_budget == 0)
        return fail(MHD_EINVAL, "bad argument");
    if (b->ndim != 3) return fail(MHD_EINVAL, "the out-of-core advance needs a 3D box");
    if (b->cfg_index.empty()) return fail(MHD_EINVAL, "no compiled kernel for this dimensionality");
    const int P = b->npatch;
    const int nx = b->pn[0], ny = b->pn[1], nz = b->pn[2];
    int64_t np3[3];
    for (int d = 0; d < 3; ++d) np3[d] = b->domain[d] / b->pn[d];
    const int64_t ppl = np3[0] * np3[1];
    const int NL = (int)np3[2];
    bool grid = ppl * NL == P;
    for (int p = 0; p < P && grid; ++p) {
        grid = b->pn[3 * p] == nx && b->pn[3 * p + 1] == ny && b->pn[3 * p + 2] == nz &&
               b->origin[3 * p] == (p % np3[0]) * nx && b->origin[3 * p + 1] == ((p / np3[0]) % np3[1]) * ny &&
               b->origin[3 * p + 2] == (p / ppl) * nz;
    }
    if (!grid) return fail(MHD_EINVAL, "the out-of-core advance needs equal patches on a grid, x fastest in patch order");
    if (ppl > 65535) return fail(MHD_EINVAL, "more than 65535 patches per z-layer");
    const PatchDev& h0 = b->hp[0];
    const int64_t pe = 8LL * h0.X * h0.Y * h0.Z;           // elements of a padded patch
    const int64_t ie = 8LL * nx * ny * nz;                 // elements of a patch's interior
    if (pe * (b->rb / 4) >= ((int64_t)1 << 31))
        return fail(MHD_EINVAL, "a patch is too large for the interior-layout copies (2^31 words)");
    const size_t PL = (size_t)(ppl * pe * b->rb), IL = (size_t)(ppl * ie * b->rb);   // bytes per layer
    // the largest chunk of L layers whose working set fits: a ring of L+2 padded layers
    // (the chunk and one layer above and below it) for U^n and one for U^{n+1}, two
    // single-layer upload stages, two chunk download stages, tables
    auto need = [&](int L) {
        const size_t tab = (size_t)L * ppl * (sizeof(PatchDev) + 27 * sizeof(int64_t) + 16 + (size_t)h0.Z * b->rb);
        return 2 * (size_t)(L + 2) * PL + 2 * IL + 2 * (size_t)L * IL + (size_t)(L + 2) * ppl * sizeof(PatchDev) + tab +
               (1 << 20);
    };
    int L = NL;
    while (L > 0 && need(L) > device_budget) --L;
    if (L == 0)
        return fail(MHD_ENOMEM, "device_budget too small: one layer of patches needs " + std::to_string(need(1)) +
                                    " bytes");
    const int K = (NL + L - 1) / L;
    const int S = L + 2;                                   // ring slots (layers)
    auto slot = [&](int g) { return ((g % S) + S) % S; };  // g: unwrapped layer index in [-1, NL]
    const bool zper_lo = b->bc[4] == MHD_BC_PERIODIC, zper_hi = b->bc[5] == MHD_BC_PERIODIC;
    const int k = b->config < 0 ? default_config(b) : b->config;
    const StepLaunch& SL = step_cfg(b, k);
    const auto& T = b->tiles[k];
    int occ = 1;
    CK(SL.occupancy(&occ));
    occ = std::max(occ, 1);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int rc = ensure_stream_pipeline(b, 4);
    if (rc) return rc;
    // ---- host tables: ring slots (scatter / gather), chunks (fill, CFL, update)
    std::vector<PatchDev> slot_tab((size_t)S * ppl);
    for (int sl = 0; sl < S; ++sl)
        for (int64_t j = 0; j < ppl; ++j) {
            PatchDev q = h0;
            q.off = ((int64_t)sl * ppl + j) * pe;
            slot_tab[(size_t)sl * ppl + j] = q;
        }
    std::vector<int64_t> ioff_layer(ppl);
    for (int64_t j = 0; j < ppl; ++j) ioff_layer[j] = j * ie;
    std::vector<PatchDev> ctab;
    std::vector<int64_t> cnb;
    std::vector<int4> ctiles;
    std::vector<int> cfirst(K), cnp(K), ctfirst(K), ctn(K);
    for (int c = 0; c < K; ++c) {
        const int z0 = c * L, z1 = std::min(NL, z0 + L);
        cfirst[c] = (int)ctab.size();
        cnp[c] = (int)((z1 - z0) * ppl);
        ctfirst[c] = (int)ctiles.size();
        for (int g = z0; g < z1; ++g)
            for (int64_t j = 0; j < ppl; ++j) {
                const int p = (int)(g * ppl + j);
                PatchDev q = b->hp[p];
                q.off = ((int64_t)slot(g) * ppl + j) * pe;
                const int local = (int)ctab.size() - cfirst[c];
                ctab.push_back(q);
                const int64_t ix = j % np3[0], iy = j / np3[0];
                for (int sz = -1; sz <= 1; ++sz)
                    for (int sy = -1; sy <= 1; ++sy)
                        for (int sx = -1; sx <= 1; ++sx) {
                            // neighbour in the ring: same layer (x, y wrapped), or the layer
                            // above / below; across an outflow box face the guard fill never
                            // reads it (clamped to the patch itself)
                            const int64_t jx = ((ix + sx) % np3[0] + np3[0]) % np3[0];
                            const int64_t jy = ((iy + sy) % np3[1] + np3[1]) % np3[1];
                            int gz = g + sz;
                            if ((gz < 0 && !zper_lo) || (gz >= NL && !zper_hi)) gz = g;
                            cnb.push_back(((int64_t)slot(gz) * ppl + jy * np3[0] + jx) * pe);
                        }
                for (int t = T.first[p]; t < T.first[p] + T.count[p]; ++t) {
                    int4 tl = T.nat_h[t];
                    tl.x = local;
                    ctiles.push_back(tl);
                }
            }
        std::stable_sort(ctiles.begin() + ctfirst[c], ctiles.end(), [](const int4& x, const int4& y) { return x.w > y.w; });
        ctn[c] = (int)ctiles.size() - ctfirst[c];
    }
    // ---- device working set (released on return)
    struct Mem {
        std::vector<void*> v;
        ~Mem() {
            for (void* x : v) cudaFree(x);
        }
        void* get(size_t n) {
            void* x = nullptr;
            if (cudaMalloc(&x, n) != cudaSuccess) return nullptr;
            v.push_back(x);
            return x;
        }
    } mem;
    char* ring = static_cast<char*>(mem.get((size_t)S * PL));
    char* ring_new = static_cast<char*>(mem.get((size_t)S * PL));
    char* in_stage[2] = {static_cast<char*>(mem.get(IL)), static_cast<char*>(mem.get(IL))};
    char* out_stage[2] = {static_cast<char*>(mem.get((size_t)L * IL)), static_cast<char*>(mem.get((size_t)L * IL))};
    PatchDev* d_slot = static_cast<PatchDev*>(mem.get(sizeof(PatchDev) * slot_tab.size()));
    int64_t* d_ioff = static_cast<int64_t*>(mem.get(sizeof(int64_t) * ppl));
    PatchDev* d_ctab = static_cast<PatchDev*>(mem.get(sizeof(PatchDev) * ctab.size()));
    int64_t* d_cnb = static_cast<int64_t*>(mem.get(sizeof(int64_t) * cnb.size()));
    int4* d_ctiles = static_cast<int4*>(mem.get(sizeof(int4) * ctiles.size()));
    void* d_part = mem.get((size_t)L * ppl * h0.Z * b->rb);
    unsigned* d_cnt = static_cast<unsigned*>(mem.get(sizeof(unsigned)));
    double* d_cdt = static_cast<double*>(mem.get(sizeof(double) * K));
    double* d_dts = static_cast<double*>(mem.get(sizeof(double) * nsteps));
    for (void* x : {(void*)ring, (void*)ring_new, (void*)in_stage[0], (void*)in_stage[1], (void*)out_stage[0],
                    (void*)out_stage[1], (void*)d_slot, (void*)d_ioff, (void*)d_ctab, (void*)d_cnb, (void*)d_ctiles,
                    d_part, (void*)d_cnt, (void*)d_cdt, (void*)d_dts})
        if (!x) return fail(MHD_ENOMEM, "cudaMalloc of the out-of-core working set failed");
    CK(cudaMemcpy(d_slot, slot_tab.data(), sizeof(PatchDev) * slot_tab.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_ioff, ioff_layer.data(), sizeof(int64_t) * ppl, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_ctab, ctab.data(), sizeof(PatchDev) * ctab.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_cnb, cnb.data(), sizeof(int64_t) * cnb.size(), cudaMemcpyHostToDevice));
    CK(cudaMemcpy(d_ctiles, ctiles.data(), sizeof(int4) * ctiles.size(), cudaMemcpyHostToDevice));
    CK(cudaMemset(d_cnt, 0, sizeof(unsigned)));
    // ---- host buffers: step s reads hbuf[r] and writes hbuf[1 - r]; the last step writes
    // host_state (an odd step count starts from a copy in host_scratch)
    char* hbuf[2] = {static_cast<char*>(host_state), static_cast<char*>(host_scratch)};
    int r = 0;
    if (nsteps % 2) {
        std::memcpy(hbuf[1], hbuf[0], (size_t)P * ie * b->rb);
        r = 1;
    }
    double dxi[3];
    int act[3];
    for (int d = 0; d < 3; ++d) {
        dxi[d] = 1.0 / b->dx[d];
        act[d] = active(b, d);
    }
    const int wpr = b->rb / 4;
    cudaEvent_t ev_up[2] = {b->ev_in[0], b->ev_in[1]}, ev_sc[2] = {b->ev_step[0], b->ev_step[1]};
    cudaEvent_t ev_ga[2] = {b->ev_in[2], b->ev_in[3]}, ev_dn[2] = {b->ev_out[0], b->ev_out[1]};
    cudaEvent_t ev_go = b->ev_step[2], ev_done = b->ev_out[2];
    int64_t nup = 0, ndown = 0;
    // the copy streams start after the work already queued on st
    CK(cudaEventRecord(ev_go, st));
    CK(cudaStreamWaitEvent(b->s_in, ev_go, 0));
    CK(cudaStreamWaitEvent(b->s_out, ev_go, 0));
    // layer g (unwrapped) of the read buffer into its ring slot: upload into a stage (copy
    // stream), scatter on st
    auto upload = [&](const char* hsrc, int g) -> int {
        const int gs = ((g % NL) + NL) % NL;
        const int u = (int)(nup++ % 2);
        CK(cudaStreamWaitEvent(b->s_in, ev_sc[u], 0));
        CK(cudaMemcpyAsync(in_stage[u], hsrc + (size_t)gs * IL, IL, cudaMemcpyHostToDevice, b->s_in));
        CK(cudaEventRecord(ev_up[u], b->s_in));
        CK(cudaStreamWaitEvent(st, ev_up[u], 0));
        interior_copy_kernel<<<dim3(nz, (unsigned)ppl), 256, 0, st>>>(
            reinterpret_cast<unsigned*>(ring), reinterpret_cast<unsigned*>(in_stage[u]), d_slot + (size_t)slot(g) * ppl,
            d_ioff, 0, (int)ppl, wpr, 1);
        ++b->launches;
        CK(cudaGetLastError());
        CK(cudaEventRecord(ev_sc[u], st));
        return MHD_OK;
    };
    // the layers of chunk c's window not left in the ring by chunk c-1
    auto load_window = [&](const char* hsrc, int c) -> int {
        const int z0 = c * L, z1 = std::min(NL, z0 + L);
        const int lo = c == 0 ? z0 - 1 : z0 + 1;
        for (int g = lo; g <= z1; ++g) {
            if ((g < 0 && !zper_lo) || (g >= NL && !zper_hi)) continue;
            const int e = upload(hsrc, g);
            if (e) return e;
        }
        return MHD_OK;
    };
    // the same going down: chunk c after chunk c+1, whose window holds c's top two layers
    auto load_window_down = [&](const char* hsrc, int c) -> int {
        const int z0 = c * L, z1 = std::min(NL, z0 + L);
        for (int g = z0 - 1; g <= z1 - 2; ++g) {
            if ((g < 0 && !zper_lo) || (g >= NL && !zper_hi)) continue;
            const int e = upload(hsrc, g);
            if (e) return e;
        }
        return MHD_OK;
    };
    for (int s = 0; s < nsteps; ++s) {
        const char* R = hbuf[r];
        char* W = hbuf[1 - r];
        // the previous step's downloads (into the buffer read now) come first
        CK(cudaStreamWaitEvent(b->s_in, ev_done, 0));
        // pass 1: guard fill + CFL rates of every chunk; dt = the smallest chunk dt
        for (int c = 0; c < K; ++c) {
            if ((rc = load_window(R, c))) return rc;
            CK(b->K->fill_cfl(ring, d_ctab + cfirst[c], h0, cnp[c], d_cnb + (size_t)cfirst[c] * 27, h0.Z, b->gamma,
                              b->courant, dxi, act, d_part, d_cnt, d_cdt + c, b->d_err, st));
            ++b->launches;
        }
        min_dt_kernel<<<1, 32, 0, st>>>(d_cdt, K, d_dts + s);
        ++b->launches;
        CK(cudaGetLastError());
        // pass 2: guard fill, update, gather and download of every chunk, last chunk first:
        // pass 1 left the last chunk's window in the ring with its guard zones filled, and
        // going down each window shares its two top layers with the one before
        for (int c = K - 1; c >= 0; --c) {
            if (c < K - 1) {
                if ((rc = load_window_down(R, c))) return rc;
                CK(b->K->fill(ring, d_ctab + cfirst[c], cnp[c], b->fg, d_cnb + (size_t)cfirst[c] * 27, h0.Z, b->d_err,
                              st));
                ++b->launches;
            }
            StepHostArgs a = step_args(b, d_dts + s, 0.0);
            a.U = ring;
            a.Unew = ring_new;
            a.patches = d_ctab + cfirst[c];
            a.tiles = d_ctiles + ctfirst[c];
            a.ntiles = ctn[c];
            a.dynamic = 1;
            CK(SL.launch(&a, std::min(ctn[c], b->nsm * occ), st));
            ++b->launches;
            const int o = (int)(ndown++ % 2);
            CK(cudaStreamWaitEvent(st, ev_dn[o], 0));
            const int z0 = c * L, z1 = std::min(NL, z0 + L);
            for (int g = z0; g < z1; ++g) {
                interior_copy_kernel<<<dim3(nz, (unsigned)ppl), 256, 0, st>>>(
                    reinterpret_cast<unsigned*>(ring_new), reinterpret_cast<unsigned*>(out_stage[o] + (size_t)(g - z0) * IL),
                    d_slot + (size_t)slot(g) * ppl, d_ioff, 0, (int)ppl, wpr, 0);
                ++b->launches;
                CK(cudaGetLastError());
            }
            CK(cudaEventRecord(ev_ga[o], st));
            CK(cudaStreamWaitEvent(b->s_out, ev_ga[o], 0));
            CK(cudaMemcpyAsync(W + (size_t)z0 * IL, out_stage[o], (size_t)(z1 - z0) * IL, cudaMemcpyDeviceToHost,
                               b->s_out));
            CK(cudaEventRecord(ev_dn[o], b->s_out));
        }
        CK(cudaEventRecord(ev_done, b->s_out));
        r = 1 - r;
    }
    CK(cudaStreamWaitEvent(st, ev_done, 0));
    std::vector<double> dts(nsteps);
    CK(cudaMemcpyAsync(dts.data(), d_dts, sizeof(double) * nsteps, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaStreamSynchronize(b->s_in));
    CK(cudaStreamSynchronize(b->s_out));
    int code = 0;
    rc = read_error(b, &code, nullptr, 0);
    if (rc) return rc;
    if (t_out) *t_out = std::accumulate(dts.begin(), dts.end(), 0.0);
    if (io_bytes) {
        io_bytes[0] = (size_t)nup * IL;
        io_bytes[1] = (size_t)nsteps * P * ie * b->rb;
    }
    return code;
} MHD_CATCH_ALL

int mhd_bunch_advance_async(mhd_bunch* b, double t_span, int max_rounds, int* rounds, int64_t* patch_updates) try {
    if (b && b->slab) return not_slab(b);
    int rc = ready(b);
    if (rc) return rc;
    if (!(t_span >= 0) || !std::isfinite(t_span) || max_rounds < 1) return fail(MHD_EINVAL, "bad argument");
    if (b->cfg_index.empty()) return fail(MHD_EINVAL, "no compiled kernel for this dimensionality");
    rc = ensure_async(b);
    if (rc) return rc;
    const int P = b->npatch;
    const int A = b->cur;
    double dxi[3];
    int act[3];
    for (int d = 0; d < 3; ++d) {
        dxi[d] = 1.0 / b->dx[d];
        act[d] = active(b, d);
    }
    const int k = b->config < 0 ? default_config(b) : b->config;
    const StepLaunch& L = step_cfg(b, k);
    const auto& T = b->tiles[k];
    int occ = 1;
    CK(L.occupancy(&occ));
    occ = std::max(occ, 1);
    if (T.n > b->atiles_cap) {
        cudaFree(b->d_atiles);
        b->d_atiles = nullptr;
        CK(cudaMalloc(&b->d_atiles, sizeof(int4) * T.n));
        b->atiles_cap = T.n;
    }
    cudaStream_t st = b->stream;
    // every patch at the common time 0 in the current buffer (slice 0)
    CK(cudaMemcpyAsync(b->d_tfirst, T.first.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(b->d_tcount, T.count.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(b->d_slice, 0, sizeof(int) * P, st));
    CK(cudaMemsetAsync(b->d_told, 0, sizeof(double) * P, st));
    CK(cudaMemsetAsync(b->d_tcur, 0, sizeof(double) * P, st));
    CK(cudaMemsetAsync(b->d_abort, 0, sizeof(unsigned), st));
    b->log_patches.clear();
    b->log_dts.clear();

    // the previous round's commit (prev < 0: none)
    auto commit = [&](int prev) -> cudaError_t {
        if (prev < 0) return cudaSuccess;
        async_commit_kernel<<<std::max(1, b->nsm), 256, 0, st>>>(
            b->d_rows_list + (size_t)prev * P, b->d_rows_n + prev, b->d_rows_dt + (size_t)prev * P,
            b->d_rows_last + (size_t)prev * P, t_span, b->d_told, b->d_tcur, b->d_slice);
        ++b->launches;
        return cudaGetLastError();
    };
    StepHostArgs a = step_args(b, nullptr, 0.0);
    a.U = b->buf[A];
    a.Unew = b->buf[1 - A];
    a.slice = b->d_slice;
    a.dt_patch = b->d_dtp;
    a.tiles = b->d_atiles;
    a.ntiles = T.n;
    a.ntiles_dev = b->d_ntiles;
    a.dynamic = 1;
    const int step_grid = std::min(T.n, b->nsm * occ);
    const int list_blocks = std::max(1, 2 * b->nsm);
    // state stride of one patch (equal patches on a regular grid, for the table-driven fill)
    const int64_t pstride = P > 1 ? b->offs[1] - b->offs[0] : (int64_t)(b->state_bytes / b->rb);

    int64_t updates = 0;
    int r = 0, prev = -1;
    std::vector<int> hn(kAsyncRows), hl;
    std::vector<double> hd;
    bool done = false;
    while (!done && r < max_rounds) {
        const int kb = std::min(kAsyncRows, max_rounds - r);
        for (int i = 0; i < kb; ++i) {
            int* row = b->d_rows_list + (size_t)i * P;
            int* nrow = b->d_rows_n + i;
            CK(commit(prev));
            async_ready_kernel<<<(P + 255) / 256, 256, 0, st>>>(P, b->d_nb_off, b->d_nb_idx, b->d_tcur, t_span,
                                                                 b->d_abort, b->d_ready);
            async_list_kernel<<<1, kSchedThreads, 0, st>>>(P, b->d_ready, b->d_tfirst, b->d_tcount, T.d_nat, row,
                                                           nrow, b->d_atiles, b->d_ntiles, b->d_rmax);
            CK(cudaGetLastError());
            // guard zones at each patch's own time, then its own CFL dt, clipped
            CK(b->K->fill_interp(b->buf[A], b->buf[1 - A], b->d_patches, P, row, P, nrow, list_blocks, b->d_slice,
                                 b->d_told, b->d_tcur, b->fg, b->d_nboff, b->hp[0].Z, pstride, b->d_err, st));
            CK(b->K->cfl_patch(b->buf[A], b->buf[1 - A], b->d_patches, row, P, nrow, list_blocks, b->d_slice,
                               b->gamma, dxi, act, b->d_rmax, b->d_err, st));
            async_clamp_kernel<<<std::max(1, (P + 255) / 256), 256, 0, st>>>(
                row, nrow, b->d_rmax, b->courant, b->d_tcur, t_span, b->d_dtp, b->d_rows_dt + (size_t)i * P,
                b->d_rows_last + (size_t)i * P, b->d_abort, b->d_err);
            CK(cudaGetLastError());
            // the update of the listed tiles, current slice -> the other, each by its own dt
            CK(L.launch(&a, step_grid, st));
            b->launches += 6;
            prev = i;
        }
        // the batch's record; an empty round means every patch has arrived (the patch at
        // the earliest time is always ready) or a round failed
        CK(cudaMemcpyAsync(hn.data(), b->d_rows_n, sizeof(int) * kb, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        int m = 0;
        while (m < kb && hn[m] > 0) ++m;
        if (m > 0) {
            hl.resize((size_t)m * P);
            hd.resize((size_t)m * P);
            CK(cudaMemcpyAsync(hl.data(), b->d_rows_list, sizeof(int) * m * P, cudaMemcpyDeviceToHost, st));
            CK(cudaMemcpyAsync(hd.data(), b->d_rows_dt, sizeof(double) * m * P, cudaMemcpyDeviceToHost, st));
            CK(cudaStreamSynchronize(st));
            for (int i = 0; i < m; ++i) {
                b->log_patches.emplace_back(hl.begin() + (size_t)i * P, hl.begin() + (size_t)i * P + hn[i]);
                b->log_dts.emplace_back(hd.begin() + (size_t)i * P, hd.begin() + (size_t)i * P + hn[i]);
                updates += hn[i];
            }
        }
        r += m;
        if (m < kb) done = true;
    }
    // commit the last round, then gather every patch's final slice into the current buffer
    CK(commit(prev));
    async_gather_kernel<<<dim3(16, std::min(P, 65535)), 256, 0, st>>>(
        static_cast<unsigned*>(b->buf[A]), static_cast<const unsigned*>(b->buf[1 - A]), b->d_patches, P,
        b->d_slice, b->rb / 4);
    CK(cudaGetLastError());
    ++b->launches;
    std::vector<double> t_cur(P);
    CK(cudaMemcpyAsync(t_cur.data(), b->d_tcur, sizeof(double) * P, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (rounds) *rounds = r;
    if (patch_updates) *patch_updates = updates;
    int code = 0;
    rc = read_error(b, &code, nullptr, 0);
    if (rc) return rc;
    if (code) return code;
    for (int p = 0; p < P; ++p)
        if (t_cur[p] < t_span) return fail(MHD_ESTATE, "max_rounds reached before every patch arrived at t_span");
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_async_round(const mhd_bunch* b, int round, int32_t* patches, double* dts, int cap, int* n) try {
    if (!b || !n) return fail(MHD_EINVAL, "NULL argument");
    if (round < 0 || round >= (int)b->log_patches.size()) return fail(MHD_EINVAL, "no such round");
    const auto& lp = b->log_patches[round];
    *n = (int)lp.size();
    if (patches || dts) {
        if (cap < *n) return fail(MHD_EINVAL, "cap smaller than the round's patch count");
        for (int i = 0; i < *n; ++i) {
            if (patches) patches[i] = lp[i];
            if (dts) dts[i] = b->log_dts[round][i];
        }
    }
    return MHD_OK;
} MHD_CATCH_ALL

int mhd_bunch_get_error(mhd_bunch* b, int* code, char* msg, size_t len) try {
    if (!b) return fail(MHD_EINVAL, "handle is NULL");
    return read_error(b, code, msg, len);
} MHD_CATCH_ALL

int mhd_bunch_launch_count(const mhd_bunch* b, int64_t* count) try {
    if (!b || !count) return fail(MHD_EINVAL, "NULL argument");
    *count = b->launches;
    return MHD_OK;
} MHD_CATCH_ALL

void mhd_bunch_destroy(mhd_bunch* b) {
    if (!b) return;
    release_graph(b);
    free_tiles(b);
    for (auto* v : {&b->ev_in, &b->ev_step, &b->ev_out})
        for (cudaEvent_t e : *v) cudaEventDestroy(e);
    if (b->s_in) cudaStreamDestroy(b->s_in);
    if (b->s_out) cudaStreamDestroy(b->s_out);
    cudaFree(b->d_slice);
    cudaFree(b->d_told);
    cudaFree(b->d_tcur);
    cudaFree(b->d_dtp);
    cudaFree(b->d_atiles);
    cudaFree(b->d_nb_off);
    cudaFree(b->d_nb_idx);
    cudaFree(b->d_tfirst);
    cudaFree(b->d_tcount);
    cudaFree(b->d_rows_list);
    cudaFree(b->d_rows_dt);
    cudaFree(b->d_rows_last);
    cudaFree(b->d_rows_n);
    cudaFree(b->d_ntiles);
    cudaFree(b->d_abort);
    cudaFree(b->d_ready);
    cudaFree(b->d_rmax);
    cudaFree(b->d_ioff);
    cudaFree(b->d_interior);
    cudaFree(b->d_patches);
    cudaFree(b->d_owner);
    cudaFree(b->d_nboff);
    cudaFree(b->d_partial_fc);
    cudaFree(b->d_slab_slots);
    cudaFree(b->d_slab_ioff);
    cudaFree(b->d_work);
    cudaFree(b->d_partial);
    cudaFree(b->d_counter);
    cudaFree(b->d_dt);
    cudaFree(b->d_dts);
    cudaFree(b->d_err);
    cudaFree(b->d_adjF);
    cudaFree(b->d_adjG);
    cudaFree(b->d_adjU);
    delete b;
}

const char* mhd_last_error(void) { return g_err.c_str(); }

}  // extern "C"

extern "C" int mhd_bunch_step_adjoint(mhd_bunch* b, double dt, const void* U_n, const void* lam_next, void* lam) try {
    if (b && b->slab) return not_slab(b);
    int rc = ready(b);
    if (rc) return rc;
    if (!U_n || !lam_next || !lam) return fail(MHD_EINVAL, "NULL argument");
    if (!(dt >= 0) || !std::isfinite(dt)) return fail(MHD_EINVAL, "dt must be finite and >= 0");
    if (b->ndim != 3) return fail(MHD_EINVAL, "the adjoint is implemented for 3D bunches");
    if (lam == lam_next || lam == U_n) return fail(MHD_EINVAL, "lam must not alias U_n or lam_next");
    const int64_t ncell = (int64_t)(b->state_bytes / b->rb) / 8;
    const size_t fbytes = (size_t)b->K->adj_fields * (size_t)ncell * b->rb;
    if (!b->d_adjF) {
        // library-owned work arrays, kept for later calls (released by mhd_bunch_destroy)
        cudaError_t e = cudaMalloc(&b->d_adjF, fbytes);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_adjG, fbytes);
        if (e == cudaSuccess) e = cudaMalloc(&b->d_adjU, b->state_bytes);
        if (e != cudaSuccess) {
            cudaFree(b->d_adjF);
            cudaFree(b->d_adjG);
            cudaFree(b->d_adjU);
            b->d_adjF = b->d_adjG = b->d_adjU = nullptr;
            return fail(MHD_ENOMEM, std::string("adjoint work arrays: ") + cudaGetErrorString(e));
        }
    }
    CK(cudaMemcpyAsync(b->d_adjU, U_n, b->state_bytes, cudaMemcpyDeviceToDevice, b->stream));
    CK(cudaMemsetAsync(b->d_adjG, 0, fbytes, b->stream));
    AdjHostArgs a;
    a.U = b->d_adjU;
    a.lam_next = lam_next;
    a.lam = lam;
    a.F = b->d_adjF;
    a.G = b->d_adjG;
    a.ncell = ncell;
    a.patches = b->d_patches;
    a.npatch = b->npatch;
    int mc = 0;
    for (const auto& q : b->hp) mc = std::max(mc, q.X * q.Y * q.Z);
    a.max_cells = mc;
    a.gamma = b->gamma;
    a.eps = hlld_eps(b->rb);
    a.dt = dt;
    for (int d = 0; d < 3; ++d) a.dxi[d] = 1.0 / b->dx[d];
    a.limiter = b->limiter;
    a.riemann = b->riemann;
    a.nboff = b->d_nboff;
    a.Zp = b->hp[0].Z;
    int n = 0;
    CK(b->K->adjoint(a, b->fg, b->d_err, b->stream, &n));
    b->launches += n;
    return MHD_OK;
} MHD_CATCH_ALL
