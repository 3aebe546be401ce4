// C ABI of the library (declared in include/lbm.h): workspace layout, set-up
// of the geometry, the per-step kernel sequence and host-side checks.
#include "lbm_internal.cuh"
#include "segments.h"

#include <cmath>
#include <ctime>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <utility>
#include <vector>

#ifndef LBM_WALL_VALUES
#define LBM_WALL_VALUES 1  // the sweep keeps the wall cells' values for the next ghost pass
#endif
#ifndef LBM_STATIC_LINKS
#define LBM_STATIC_LINKS 1  // 1: static-wall links regrouped by direction for the ghost pass
#endif
#ifndef LBM_SEG_SECTOR
#define LBM_SEG_SECTOR 1  // 1: sweep segments complete the 32-byte sectors at the ends of fluid runs
#endif

namespace lbmgb {
size_t stats_partials_doubles();

namespace {

constexpr size_t ALIGN = 256;

struct Layout {
    size_t off = 0;
    size_t take(size_t bytes) {
        const size_t o = off;
        off += (bytes + ALIGN - 1) / ALIGN * ALIGN;
        return o;
    }
};

struct Plan {
    long long N, max_sites, max_links, max_markers;
    int max_np, nblk;
    size_t fA, fB, flags, owner, aux;
    size_t site_cell, site_first, site_mask, sup_ru, sup_F, sup_Fp;
    size_t link_cell, link_pid, link_dir, link_scheme, link_q, link_dP, link_dT;
    size_t blk_sites, blk_links, counts, status, seg, slink, slink_rank, slink4, seg_bnd, bvals, wrec, gidx, gvals, wcoef, wlane, pair_items, pair_wall, wslot, refill;
    long long max_refill;
    long long max_seg;
    size_t xy_start, xy_j, xy_w, it_k, it_w;
    int max_ring;
    long long max_xy;
    size_t pX, pXold, pU, pW, pR, pmass, pinertia, pFh, pTh, pFprev, pTprev, pFc, pIu, pIr, phas, pXf, sn_list;
    size_t mX, mUnit, mdV, mUd, mFaccR, mFacc, mFr, mB, mE, mpid, mfirst;
    size_t rho_f, u_f, partials, near_key;
    size_t cl_w, cl_pk, cl_X, cl_Y, cl_cells, cl_eps;
    long long max_cl;
    size_t q27_colmask, q27_hmask, q27_coef;
    size_t total;
};

bool make_plan(const lbm_grid *g, Plan &P) {
    if (!g || g->nx < 4 || g->ny < 4 || g->nz < 1) return false;
    if (g->storage < LBM_F64 || g->storage > LBM_BF16S) return false;
    if (g->rates != LBM_RATES_SRT && g->rates != LBM_RATES_DHUMIERES) return false;
    if (g->max_particles < 0 || g->max_links < 0 || g->max_markers < 0 || g->max_sites < 0) return false;
    if (g->max_particles > LBM_MAX_PARTICLES) return false;
    if (g->lattice != 0 && g->lattice != 19 && g->lattice != 27) return false;
    // D3Q27: periodic box, BGK, FP64 or FP32 storage
    if (g->lattice == 27 && (g->rates != LBM_RATES_SRT || (g->storage != LBM_F64 && g->storage != LBM_F32)))
        return false;
    const long long N = (long long)g->nx * g->ny * g->nz;
    if (N >= (1LL << 31) - 4096) return false;
    P.N = N;
    P.max_np = g->max_particles;
    P.max_links = g->max_links > 0 ? g->max_links : N / 4 + 65536;
    P.max_sites = g->max_sites > 0 ? g->max_sites : N / 4 + 65536;
    const long long ring = 8LL * (g->nx + g->ny) * g->nz;
    P.max_markers = g->max_markers > 0 ? g->max_markers : (long long)P.max_np * 260 + ring;
    P.nblk = (int)((N + 1023) / 1024);
    const size_t sb = storage_bytes(g->storage);
    const size_t n = (size_t)N, ms = (size_t)P.max_sites, ml = (size_t)P.max_links, mm = (size_t)P.max_markers;
    const size_t np = (size_t)(P.max_np > 0 ? P.max_np : 1);
    Layout L;
    const size_t nq = g->lattice == 27 ? 27 : 19;
    P.fA = L.take(nq * n * sb);
    P.fB = L.take(nq * n * sb);
    P.flags = L.take(n + 8);
    P.owner = L.take(4 * n);
    P.aux = L.take(4 * n);
    P.site_cell = L.take(4 * ms);
    P.site_first = L.take(4 * ms);
    P.site_mask = L.take(4 * ms);
    P.sup_ru = L.take(32 * ms);
    P.sup_F = L.take(24 * ms);
    P.sup_Fp = L.take(24 * ms);
    P.link_cell = L.take(4 * ml);
    P.link_pid = L.take(4 * ml);
    P.link_dir = L.take(ml);
    P.link_scheme = L.take(ml);
    P.link_q = L.take(8 * ml);
    P.link_dP = L.take(24 * ml);
    P.link_dT = L.take(24 * ml);
    P.max_xy = 64LL * (g->nx + g->ny);
    P.xy_start = L.take(4 * ((size_t)g->nx * g->ny + 1));
    P.xy_j = L.take(4 * (size_t)P.max_xy);
    P.xy_w = L.take(8 * (size_t)P.max_xy);
    P.max_ring = 4 * (g->nx + g->ny);
    P.it_k = L.take(4 * 16 * (size_t)P.max_ring);
    P.it_w = L.take(8 * 16 * (size_t)P.max_ring);
    P.max_seg = (long long)g->ny * g->nz * ((g->nx + 31) / 32 + 1);
    P.seg = L.take(16 * (size_t)P.max_seg);
    P.slink = L.take(8 * ml);
    P.slink_rank = L.take(4 * ml);
    P.slink4 = L.take(16 * ml);
    P.seg_bnd = L.take(8 * (size_t)P.max_seg);
    P.bvals = L.take(19 * sb * ms);
    P.wrec = L.take(8 * ms);
    P.gidx = L.take(4 * ml);
    P.gvals = L.take(sb * ml);
    P.wcoef = L.take(8 * ml);
    P.wlane = L.take(2 * ml);
    P.pair_items = L.take(16 * (size_t)P.max_seg);
    P.pair_wall = L.take(16 * (size_t)P.max_seg);
    P.wslot = L.take(2 * ml);
    P.blk_sites = L.take(8 * (size_t)P.nblk);
    P.blk_links = L.take(8 * (size_t)P.nblk);
    P.counts = L.take(64);
    P.max_refill = 256LL * (P.max_np > 0 ? P.max_np : 1);
    P.refill = L.take(8 * (size_t)P.max_refill);
    P.status = L.take(16);
    P.pX = L.take(24 * np);
    P.pXold = L.take(24 * np);
    P.pU = L.take(24 * np);
    P.pW = L.take(24 * np);
    P.pR = L.take(8 * np);
    P.pmass = L.take(8 * np);
    P.pinertia = L.take(8 * np);
    P.pFh = L.take(24 * np);
    P.pTh = L.take(24 * np);
    P.pFprev = L.take(24 * np);
    P.pTprev = L.take(24 * np);
    P.pFc = L.take(48 * np);
    P.pIu = L.take(24 * np);
    P.pIr = L.take(24 * np);
    P.phas = L.take(4 * np);
    P.pXf = L.take(16 * np);
    P.sn_list = L.take(4 * ml);
    P.mX = L.take(24 * mm);
    P.mUnit = L.take(24 * mm);
    P.mdV = L.take(8 * mm);
    P.mUd = L.take(24 * mm);
    P.mFaccR = L.take(24 * mm);
    P.mFacc = L.take(24 * mm);
    P.mFr = L.take(24 * mm);
    P.mB = L.take(12 * mm);
    P.mE = L.take(24 * mm);
    P.mpid = L.take(4 * mm);
    P.mfirst = L.take(4 * (np + 1));
    P.rho_f = L.take(8 * n);
    P.u_f = L.take(24 * n);
    P.partials = L.take(8 * stats_partials_doubles());
    P.near_key = L.take(8 * n);
    P.max_cl = P.max_np > 0 ? 1500LL * P.max_np : 0;
    P.cl_w = L.take(4 * 14409);
    P.cl_pk = L.take(mlp_pack_bytes());
    P.cl_X = L.take(4 * 85 * (size_t)P.max_cl);
    P.cl_Y = L.take(4 * 9 * (size_t)P.max_cl);
    P.cl_cells = L.take(4 * (size_t)P.max_cl);
    P.cl_eps = L.take(P.max_cl > 0 ? 4 * n : 0);
    P.q27_colmask = L.take(g->lattice == 27 ? 4 * (size_t)g->nx * g->ny : 0);
    P.q27_hmask = L.take(g->lattice == 27 ? 4 * (size_t)g->nx * g->ny : 0);
    P.q27_coef = L.take(g->lattice == 27 ? 2 * sb * 27 * (size_t)g->nx * g->ny : 0);
    P.total = L.off;
    return true;
}

lbm_status fail(Ctx &c, lbm_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c.err, sizeof(c.err), fmt, ap);
    va_end(ap);
    return s;
}

lbm_status cuda_fail(Ctx &c, cudaError_t e, const char *where) {
    c.broken = true;
    return fail(c, LBM_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);     \
    } while (0)

__global__ void fill_owner(int *p, long long n) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = NO_OWNER;
}

template <typename R>
__global__ void dense_ibm_force(double *out, const R *sup_F, const int *site_cell, const long long *counts,
                                long long max_sites, long long N) {
    const long long ns = counts[0] < max_sites ? counts[0] : max_sites;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < ns; s += (long long)gridDim.x * blockDim.x) {
        const int c = site_cell[s];
        out[c] = sup_F[3 * s];
        out[N + c] = sup_F[3 * s + 1];
        out[2 * N + c] = sup_F[3 * s + 2];
    }
}

template <int S>
__global__ void plane_to_f64(const void *src, double *dst, long long N, int i) {
    typedef typename Store<S>::T T;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const T *p = (const T *)src + (size_t)i * N + c;
    double v;
    if (S == LBM_F64) v = *(const double *)p;
    else if (S == LBM_F32) v = *(const float *)p;
    else if (S == LBM_F16S) v = (double)__half2float(*(const __half *)p) / (double)F16_SCALE;
    else v = (double)__bfloat162float(*(const __nv_bfloat16 *)p);
    dst[c] = v + wgt(i);
}
template <int S>
__global__ void f64_to_plane(void *dst, const double *src, long long N, int i) {
    typedef typename Store<S>::T T;
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    Store<S>::st((T *)dst + (size_t)i * N + c, typename Store<S>::R(src[c] - wgt(i)));
}

cudaError_t plane_copy(Ctx &c, int i, bool to_f64) {
    const unsigned nb = (unsigned)((c.N + 255) / 256);
#define PC(S)                                                                                 \
    if (to_f64) plane_to_f64<S><<<nb, 256, 0, c.stream>>>(c.fA, c.rho_f, c.N, i);            \
    else f64_to_plane<S><<<nb, 256, 0, c.stream>>>(c.fA, c.rho_f, c.N, i);
    switch (c.storage) {
    case LBM_F64: PC(LBM_F64); break;
    case LBM_F32: PC(LBM_F32); break;
    case LBM_F16S: PC(LBM_F16S); break;
    default: PC(LBM_BF16S); break;
    }
#undef PC
    return cudaGetLastError();
}

// Check the status word copied by the last asynchronous check (bounded
// host wait: polls the event, gives up after the context's wait limit).
lbm_status check_status(Ctx &c, bool wait) {
    if (!c.status_pending) return LBM_OK;
    const double timeout_s = c.wait_limit_s;
    cudaError_t q = cudaEventQuery(c.ev_status);
    if (q == cudaErrorNotReady) {
        if (!wait) return LBM_OK;
        // bounded wait
        const long long sleeps = (long long)(timeout_s * 1000.0);
        for (long long k = 0; k < sleeps; k++) {
            q = cudaEventQuery(c.ev_status);
            if (q != cudaErrorNotReady) break;
            struct timespec ts = {0, 1000000};
            nanosleep(&ts, nullptr);
        }
        if (q == cudaErrorNotReady) return fail(c, LBM_ETIMEOUT, "stream did not finish within %g s", timeout_s);
    }
    if (q != cudaSuccess) return cuda_fail(c, q, "status event");
    c.status_pending = false;
    const unsigned st = *c.h_status;
    if (st & 1u) {
        c.broken = true;
        return fail(c, LBM_EUNSTABLE, "watchdog: NaN/Inf, rho outside [0.5,2] or |u| > 0.3 before step %lld",
                    c.step);
    }
    if (st & 2u) {
        c.broken = true;
        return fail(c, LBM_ENOMEM, "site or link capacity exceeded (max_sites %lld, max_links %lld)", c.max_sites,
                    c.max_links);
    }
    return LBM_OK;
}

lbm_status enqueue_status(Ctx &c) {
    CK(cudaMemcpyAsync(c.h_status, c.d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaEventRecord(c.ev_status, c.stream));
    c.status_pending = true;
    return LBM_OK;
}

lbm_status sync_all(Ctx &c) {
    lbm_status s = enqueue_status(c);
    if (s != LBM_OK) return s;
    s = check_status(c, true);
    if (s != LBM_OK) return s;
    long long cnt[2];
    CK(cudaMemcpyAsync(cnt, c.d_counts, sizeof(cnt), cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    c.nsites = cnt[0];
    c.nlinks = cnt[1];
    return LBM_OK;
}

void set_rates(Ctx &c) {
    const double om = 1.0 / c.tau;
    Rates &r = c.rt;
    r.d_nu = om;
    if (c.rates == LBM_RATES_DHUMIERES) {
        r.d_e = 1.19;
        r.d_eps = 1.4;
        r.d_q = 1.2;
        r.d_pi = 1.4;
        r.d_m = 1.98;
    } else {
        r.d_e = r.d_eps = r.d_q = r.d_pi = r.d_m = om;
    }
    r.s_nu = (float)r.d_nu;
    r.s_e = (float)r.d_e;
    r.s_eps = (float)r.d_eps;
    r.s_q = (float)r.d_q;
    r.s_pi = (float)r.d_pi;
    r.s_m = (float)r.d_m;
}

struct ProfRec {
    int group;
    cudaEvent_t a, b;
};
struct Prof {
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> pool;
    double ms[LBM_NGROUPS];
    long long spans[LBM_NGROUPS];
    long long launches0[LBM_NGROUPS];
};

// event recorded on the stream now (nullptr when profiling is off)
cudaEvent_t pmark(Ctx &c) {
    if (!c.prof_on) return nullptr;
    Prof *P = (Prof *)c.prof;
    cudaEvent_t e;
    if (!P->pool.empty()) {
        e = P->pool.back();
        P->pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        return nullptr;
    }
    cudaEventRecord(e, c.stream);
    return e;
}
void pspan(Ctx &c, int g, cudaEvent_t a, cudaEvent_t b) {
    if (!a || !b) return;
    ((Prof *)c.prof)->recs.push_back({g, a, b});
}

int marker_count(double RL) { return (int)std::floor(M_PI / 3.0 * (12.0 * RL * RL + 1.0) + 0.5); }

// Peskin (2002) 4-point kernel, host copy for the static pipe weights
// weight tables are read in the storage's arithmetic type (FP32 unless the
// populations are FP64): converted once here, not per use on the device
cudaError_t upload_weights(const Ctx &c, void *dst, const std::vector<double> &w) {
    if (w.empty()) return cudaSuccess;
    if (c.storage == LBM_F64) return cudaMemcpy(dst, w.data(), sizeof(double) * w.size(), cudaMemcpyHostToDevice);
    std::vector<float> f(w.begin(), w.end());
    return cudaMemcpy(dst, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice);
}

double peskin_host(double r) {
    const double a = std::fabs(r);
    if (a <= 1.0) return (3.0 - 2.0 * a + std::sqrt(1.0 + 4.0 * a - 4.0 * a * a)) * 0.125;
    if (a <= 2.0) return (5.0 - 2.0 * a - std::sqrt(-7.0 + 12.0 * a - 4.0 * a * a)) * 0.125;
    return 0.0;
}

// Lagrangian markers (Sec. 2.1: marker volume close to the cell volume).
// Spheres: golden-spiral points at R_L = R - r_d, dV = pi (12 R_L^2 + 1) / (3 N_L).
// Pipe: a ring of round(2 pi R_L) points at R_L = R + r_d in every z plane.
lbm_status build_markers(Ctx &c) {
    const double rd = c.rd;
    std::vector<double> unit, X, dV;
    std::vector<int> pid, first;
    if (c.has_pipe) {
        const double RL = c.pipe_R + rd;
        const int nc = (int)std::floor(2.0 * M_PI * RL + 0.5);
        std::vector<double> rx(nc), ry(nc);
        for (int j = 0; j < nc; j++) {
            const double th = 2.0 * M_PI * j / nc;
            rx[j] = c.pipe_cx + RL * std::cos(th);
            ry[j] = c.pipe_cy + RL * std::sin(th);
        }
        for (int z = 0; z < c.nz; z++)
            for (int j = 0; j < nc; j++) {
                X.push_back(rx[j]);
                X.push_back(ry[j]);
                X.push_back((double)z);
                dV.push_back(2.0 * M_PI * RL / nc);
                pid.push_back(-1);
            }
        unit.assign(X.size(), 0.0);
        // per (x, y) column: the ring markers covering it and their x-y weights
        const long long nxy = (long long)c.nx * c.ny;
        std::vector<std::vector<std::pair<int, double>>> lists((size_t)nxy);
        for (int j = 0; j < nc; j++) {
            const int bx = (int)std::floor(rx[j]) - 1, by = (int)std::floor(ry[j]) - 1;
            for (int ky = 0; ky < 4; ky++)
                for (int kx = 0; kx < 4; kx++) {
                    const double w = peskin_host((double)(bx + kx) - rx[j]) * peskin_host((double)(by + ky) - ry[j]);
                    if (w == 0.0) continue;
                    const int xw = ((bx + kx) % c.nx + c.nx) % c.nx, yw = ((by + ky) % c.ny + c.ny) % c.ny;
                    lists[(size_t)xw + (size_t)c.nx * yw].push_back({j, w});
                }
        }
        std::vector<int> st((size_t)nxy + 1), jj;
        std::vector<double> ww;
        for (long long k = 0; k < nxy; k++) {
            st[k] = (int)jj.size();
            for (auto &e : lists[k]) {
                jj.push_back(e.first);
                ww.push_back(e.second);
            }
        }
        st[nxy] = (int)jj.size();
        if ((long long)jj.size() > c.pipe_max_xy) return fail(c, LBM_ENOMEM, "pipe marker lists exceed capacity");
        CK(cudaMemcpy(c.pipe_xy_start, st.data(), sizeof(int) * st.size(), cudaMemcpyHostToDevice));
        if (!jj.empty()) {
            CK(cudaMemcpy(c.pipe_xy_j, jj.data(), sizeof(int) * jj.size(), cudaMemcpyHostToDevice));
            CK(upload_weights(c, c.pipe_xy_w, ww));
        }
        c.pipe_nc = nc;
        c.pipe_dV = 2.0 * M_PI * RL / nc;
    } else {
        std::vector<double> R(c.np);
        CK(cudaMemcpy(R.data(), c.R, sizeof(double) * c.np, cudaMemcpyDeviceToHost));
        const double ga = M_PI * (3.0 - std::sqrt(5.0));
        for (int p = 0; p < c.np; p++) {
            first.push_back((int)pid.size());
            const double RL = R[p] - rd;
            const int n = marker_count(RL);
            for (int l = 0; l < n; l++) {
                const double zz = 1.0 - (2.0 * l + 1.0) / n;
                const double rr = std::sqrt(1.0 - zz * zz);
                const double th = ga * l;
                unit.push_back(RL * rr * std::cos(th));
                unit.push_back(RL * rr * std::sin(th));
                unit.push_back(RL * zz);
                dV.push_back(M_PI * (12.0 * RL * RL + 1.0) / (3.0 * n));
                pid.push_back(p);
            }
        }
        first.push_back((int)pid.size());
        X.assign(unit.size(), 0.0);
    }
    const long long nm = (long long)pid.size();
    if (nm > c.max_markers) return fail(c, LBM_ENOMEM, "markers %lld exceed capacity %lld", nm, c.max_markers);
    c.nm = nm;
    if (nm > 0) {
        CK(cudaMemcpyAsync(c.mUnit, unit.data(), sizeof(double) * unit.size(), cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemcpyAsync(c.mX, X.data(), sizeof(double) * X.size(), cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemcpyAsync(c.mdV, dV.data(), sizeof(double) * dV.size(), cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemcpyAsync(c.mpid, pid.data(), sizeof(int) * pid.size(), cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemsetAsync(c.mFacc, 0, sizeof(double) * 3 * nm, c.stream));
    }
    if (!first.empty())
        CK(cudaMemcpyAsync(c.m_first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return LBM_OK;
}

// The pipe's support set is the same in every z plane and the sites are
// listed in cell order, so site (x, y, z) = z * S_p + k(x, y). For each ring
// marker, its 4 x 4 column box gives up to 16 (k, x-y weight) entries; the
// interpolation then needs no per-node lookup. Left unbuilt (pipe_sp = 0)
// when the site list is not of that form.
lbm_status build_pipe_interp(Ctx &c) {
    c.pipe_sp = 0;
    const long long ns = c.nsites;
    if (ns <= 0 || ns % c.nz != 0 || c.pipe_nc <= 0 || c.pipe_nc > c.pipe_max_ring || ns > c.max_sites) return LBM_OK;
    const long long sp = ns / c.nz, nxy = (long long)c.nx * c.ny;
    std::vector<int> cell((size_t)ns);
    CK(cudaMemcpy(cell.data(), c.site_cell, sizeof(int) * ns, cudaMemcpyDeviceToHost));
    for (long long i = 0; i < ns; i++)
        if ((long long)cell[i] - (i / sp) * nxy != (long long)cell[i % sp]) return LBM_OK;  // not plane-invariant
    std::vector<int> local((size_t)nxy, -1);
    for (long long k = 0; k < sp; k++) local[cell[k]] = (int)k;
    const double RL = c.pipe_R + c.rd;
    const int nc = c.pipe_nc;
    std::vector<int> tk(16 * (size_t)nc, 0);
    std::vector<double> tw(16 * (size_t)nc, 0.0);
    for (int j = 0; j < nc; j++) {
        const double th = 2.0 * M_PI * j / nc;
        const double rx = c.pipe_cx + RL * std::cos(th), ry = c.pipe_cy + RL * std::sin(th);
        const int bx = (int)std::floor(rx) - 1, by = (int)std::floor(ry) - 1;
        for (int ky = 0; ky < 4; ky++)
            for (int kx = 0; kx < 4; kx++) {
                const int xw = ((bx + kx) % c.nx + c.nx) % c.nx, yw = ((by + ky) % c.ny + c.ny) % c.ny;
                const int k = local[(size_t)xw + (size_t)c.nx * yw];
                const double w = peskin_host((double)(bx + kx) - rx) * peskin_host((double)(by + ky) - ry);
                tk[16 * (size_t)j + 4 * ky + kx] = k < 0 ? 0 : k;
                tw[16 * (size_t)j + 4 * ky + kx] = k < 0 ? 0.0 : w;  // no site: no contribution
            }
    }
    CK(cudaMemcpy(c.pipe_it_k, tk.data(), sizeof(int) * tk.size(), cudaMemcpyHostToDevice));
    CK(upload_weights(c, c.pipe_it_w, tw));
    c.pipe_sp = (int)sp;
    return LBM_OK;
}

lbm_status arm(Ctx &c, int bc) {
    c.armed_bc = bc;
    if (bc == LBM_BC_IBM_U || bc == LBM_BC_IBM_B) {
        c.rd = bc == LBM_BC_IBM_B ? 0.4 : 0.0;
        if (c.has_pipe || c.np > 0) {
            lbm_status s = build_markers(c);
            if (s != LBM_OK) return s;
            CK(launch_markers_place(c));
            CK(launch_marker_offsets(c));
            CK(launch_ibm_rigid_overwrite(c));
            CK(launch_ibm_particle_sums(c, true));
        }
        // the spreading accumulates into this buffer and every pass clears
        // the slots it used; it must start at zero
        CK(cudaMemsetAsync(c.sup_Fp, 0, sizeof(double) * 3 * (size_t)c.max_sites, c.stream));
        CK(launch_support_mark(c));
        CK(build_sites(c, 2));
        lbm_status s = sync_all(c);
        if (s != LBM_OK) return s;
        c.nsites_hint = c.nsites;
        if (c.has_pipe && c.np == 0) {
            s = build_pipe_interp(c);
            if (s != LBM_OK) return s;
        }
    }
    return LBM_OK;
}

}  // namespace

cudaEvent_t prof_event(Ctx &c) { return pmark(c); }
void prof_span(Ctx &c, int g, cudaEvent_t a, cudaEvent_t b) { pspan(c, g, a, b); }
}  // namespace lbmgb

using namespace lbmgb;

extern "C" {

size_t lbm_workspace_bytes(const lbm_grid *grid) {
    Plan P;
    if (!make_plan(grid, P)) return 0;
    return P.total;
}

lbm_status lbm_create(const lbm_grid *grid, double tau, const double force[3], void *dev_workspace, size_t bytes,
                      void *cuda_stream, lbm_ctx **out) {
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    Plan P;
    if (!make_plan(grid, P) || !(tau > 0.5) || !dev_workspace || ((uintptr_t)dev_workspace % ALIGN) != 0)
        return LBM_EINVAL;
    if (bytes < P.total) return LBM_ENOMEM;
    lbm_ctx *h = new (std::nothrow) lbm_ctx;
    if (!h) return LBM_ENOMEM;
    memset(&h->c, 0, sizeof(Ctx));
    Ctx &c = h->c;
    c.g = *grid;
    c.nx = grid->nx;
    c.ny = grid->ny;
    c.nz = grid->nz;
    c.N = P.N;
    c.tau = tau;
    for (int d = 0; d < 3; d++) c.F[d] = force ? force[d] : 0.0;
    c.storage = grid->storage;
    c.rates = grid->rates;
    c.q = grid->lattice == 27 ? 27 : 19;
    set_rates(c);
    c.stream = (cudaStream_t)cuda_stream;
    c.ws = (char *)dev_workspace;
    c.ws_bytes = bytes;
    char *b = c.ws;
    c.fA = b + P.fA;
    c.fB = b + P.fB;
    c.flags = (uint8_t *)(b + P.flags);
    c.owner = (int *)(b + P.owner);
    c.aux = (int *)(b + P.aux);
    c.max_sites = P.max_sites;
    c.site_cell = (int *)(b + P.site_cell);
    c.site_first = (int *)(b + P.site_first);
    c.site_mask = (unsigned *)(b + P.site_mask);
    c.sup_ru = b + P.sup_ru;
    c.sup_F = b + P.sup_F;
    c.sup_Fp = b + P.sup_Fp;
    c.max_links = P.max_links;
    c.link_cell = (int *)(b + P.link_cell);
    c.link_pid = (int *)(b + P.link_pid);
    c.link_dir = (int8_t *)(b + P.link_dir);
    c.link_scheme = (int8_t *)(b + P.link_scheme);
    c.link_q = (double *)(b + P.link_q);
    c.link_dP = b + P.link_dP;
    c.link_dT = b + P.link_dT;
    c.pipe_xy_start = (int *)(b + P.xy_start);
    c.pipe_xy_j = (int *)(b + P.xy_j);
    c.pipe_xy_w = b + P.xy_w;
    c.pipe_it_k = (int *)(b + P.it_k);
    c.pipe_it_w = b + P.it_w;
    c.pipe_max_ring = P.max_ring;
    c.pipe_sp = 0;
    c.pipe_max_xy = P.max_xy;
    c.seg = (uint4 *)(b + P.seg);
    c.slink = (uint2 *)(b + P.slink);
    c.static_links = 0;
    c.slink_rank = (int *)(b + P.slink_rank);
    c.slink4 = (uint4 *)(b + P.slink4);
    c.seg_bnd = (uint2 *)(b + P.seg_bnd);
    c.bvals = b + P.bvals;
    c.wrec = (uint2 *)(b + P.wrec);
    c.gidx = (int *)(b + P.gidx);
    c.gvals = b + P.gvals;
    c.wcoef = (uint2 *)(b + P.wcoef);
    c.wlane = (unsigned short *)(b + P.wlane);
    c.pair_items = (uint4 *)(b + P.pair_items);
    c.pair_wall = (uint4 *)(b + P.pair_wall);
    c.wslot = (unsigned short *)(b + P.wslot);
    c.pair_ready = 0;
    c.wcoef_ready = 0;
    c.max_bvals = P.max_sites;
    c.bvals_ready = 0;
    c.bvals_valid = 0;
    c.max_seg = P.max_seg;
    c.nseg = 0;
    c.nblk = P.nblk;
    c.blk_sites = (long long *)(b + P.blk_sites);
    c.blk_links = (long long *)(b + P.blk_links);
    c.d_counts = (long long *)(b + P.counts);
    c.refill_list = (int *)(b + P.refill);
    c.refill_pid = c.refill_list + P.max_refill;
    c.max_refill = P.max_refill;
    c.d_status = (unsigned *)(b + P.status);
    c.max_np = P.max_np;
    c.X = (double *)(b + P.pX);
    c.Xold = (double *)(b + P.pXold);
    c.U = (double *)(b + P.pU);
    c.W = (double *)(b + P.pW);
    c.R = (double *)(b + P.pR);
    c.mass = (double *)(b + P.pmass);
    c.inertia = (double *)(b + P.pinertia);
    c.Fh = (double *)(b + P.pFh);
    c.Th = (double *)(b + P.pTh);
    c.Fprev = (double *)(b + P.pFprev);
    c.Tprev = (double *)(b + P.pTprev);
    c.Fc = (double *)(b + P.pFc);
    c.Iu = (double *)(b + P.pIu);
    c.Ir = (double *)(b + P.pIr);
    c.has_prev = (int *)(b + P.phas);
    c.Xf = (float4 *)(b + P.pXf);
    c.sn_list = (int *)(b + P.sn_list);
    c.max_markers = P.max_markers;
    c.mX = (double *)(b + P.mX);
    c.mUnit = (double *)(b + P.mUnit);
    c.mdV = (double *)(b + P.mdV);
    c.mUd = b + P.mUd;
    c.mFaccR = b + P.mFaccR;
    c.mFacc = (double *)(b + P.mFacc);
    c.mFr = b + P.mFr;
    c.mB = (int *)(b + P.mB);
    c.mE = b + P.mE;
    c.mpid = (int *)(b + P.mpid);
    c.m_first = (int *)(b + P.mfirst);
    c.rho_f = (double *)(b + P.rho_f);
    c.u_f = (double *)(b + P.u_f);
    c.partials = (double *)(b + P.partials);
    c.near_key = (unsigned long long *)(b + P.near_key);
    c.cl_w = (float *)(b + P.cl_w);
    c.cl_pk = b + P.cl_pk;
    c.cl_X = (float *)(b + P.cl_X);
    c.cl_Y = (float *)(b + P.cl_Y);
    c.cl_cells = (int *)(b + P.cl_cells);
    c.cl_eps = (float *)(b + P.cl_eps);
    c.max_cl = P.max_cl;
    c.q27_colmask = (unsigned *)(b + P.q27_colmask);
    c.q27_hmask = (unsigned *)(b + P.q27_hmask);
    c.q27_coef = (void *)(b + P.q27_coef);
    c.armed_bc = -1;
    c.wait_limit_s = 600.0;
    c.pipe_cx = 0.5 * (c.nx - 1);
    c.pipe_cy = 0.5 * (c.ny - 1);
    auto bad = [&](cudaError_t e, const char *w) {
        cuda_fail(c, e, w);
        if (c.h_status) cudaFreeHost(c.h_status);
        delete h;
        return LBM_ECUDA;
    };
    cudaError_t e;
    if ((e = cudaMallocHost((void **)&c.h_status, sizeof(unsigned))) != cudaSuccess) {
        c.h_status = nullptr;
        return bad(e, "cudaMallocHost");
    }
    *c.h_status = 0;
    if ((e = cudaEventCreateWithFlags(&c.ev_status, cudaEventDisableTiming)) != cudaSuccess) return bad(e, "event");
    const size_t sb = storage_bytes(c.storage);
    // rest state: g = f - w = 0 in every storage format
    if ((e = cudaMemsetAsync(c.fA, 0, c.q * (size_t)c.N * sb, c.stream)) != cudaSuccess) return bad(e, "memset");
    if ((e = cudaMemsetAsync(c.fB, 0, c.q * (size_t)c.N * sb, c.stream)) != cudaSuccess) return bad(e, "memset");
    if ((e = cudaMemsetAsync(c.flags, 0, (size_t)c.N + 8, c.stream)) != cudaSuccess) return bad(e, "memset");
    if ((e = cudaMemsetAsync(c.aux, 0xff, 4 * (size_t)c.N, c.stream)) != cudaSuccess) return bad(e, "memset");
    if ((e = cudaMemsetAsync(c.d_counts, 0, 64, c.stream)) != cudaSuccess) return bad(e, "memset");
    if ((e = cudaMemsetAsync(c.d_status, 0, 16, c.stream)) != cudaSuccess) return bad(e, "memset");
    fill_owner<<<(unsigned)((c.N + 255) / 256), 256, 0, c.stream>>>(c.owner, c.N);
    if ((e = cudaGetLastError()) != cudaSuccess) return bad(e, "fill");
    if ((e = cudaStreamSynchronize(c.stream)) != cudaSuccess) return bad(e, "sync");
    *out = h;
    return LBM_OK;
}

#define CTX_CHECK(h)                                       \
    if (!(h)) return LBM_EINVAL;                           \
    Ctx &c = (h)->c;

lbm_status lbm_init_velocity(lbm_ctx *h, const double *u_host, double rho0) {
    CTX_CHECK(h);
    if (!u_host || !(rho0 > 0)) return fail(c, LBM_EINVAL, "bad velocity field or rho0");
    if (c.broken || c.armed_bc >= 0) return fail(c, LBM_ESTATE, "init_velocity only before the first step");
    c.bvals_valid = 0;
    CK(cudaMemcpyAsync(c.u_f, u_host, sizeof(double) * 3 * c.N, cudaMemcpyHostToDevice, c.stream));
    if (c.q == 27) CK(launch_q27_init(c, c.u_f, rho0));
    else CK(launch_init_equilibrium(c, c.u_f, rho0));
    CK(cudaStreamSynchronize(c.stream));
    return LBM_OK;
}

lbm_status lbm_set_populations(lbm_ctx *h, const double *f_host) {
    CTX_CHECK(h);
    if (!f_host) return fail(c, LBM_EINVAL, "null populations");
    if (c.broken) return fail(c, LBM_ESTATE, "context unusable after an error");
    c.bvals_valid = 0;
    for (int i = 0; i < c.q; i++) {
        CK(cudaMemcpyAsync(c.rho_f, f_host + (size_t)i * c.N, sizeof(double) * c.N, cudaMemcpyHostToDevice, c.stream));
        if (c.q == 27) CK(q27_plane_copy(c, i, false));
        else CK(plane_copy(c, i, false));
    }
    CK(cudaStreamSynchronize(c.stream));
    return LBM_OK;
}

lbm_status lbm_set_pipe(lbm_ctx *h, double radius) {
    CTX_CHECK(h);
    if (c.broken || c.armed_bc >= 0 || c.np > 0 || c.has_pipe) return fail(c, LBM_ESTATE, "geometry already set");
    if (!(radius > 1.0) || radius > 0.5 * (c.nx < c.ny ? c.nx : c.ny)) return fail(c, LBM_EINVAL, "bad pipe radius");
    if (c.q == 27) {
        // D3Q27: the pipe wall by linear IBB inside the sweep (q27.cu)
        c.has_pipe = 1;
        c.pipe_R = radius;
        CK(launch_pipe_flags(c));
        std::vector<unsigned> mask;
        q27_pipe_colmask(c, mask);
        CK(cudaMemcpy(c.q27_colmask, mask.data(), sizeof(unsigned) * mask.size(), cudaMemcpyHostToDevice));
        CK(launch_q27_coef(c));
        // no fluid column on an x or y face: the sweep addresses pulls by plane pointers
        c.pipe_nowrap = 1;
        for (int y = 0; y < c.ny; y++)
            for (int x = 0; x < c.nx; x++)
                if (!(mask[(size_t)x + (size_t)c.nx * y] & 1u) && (x == 0 || x == c.nx - 1 || y == 0 || y == c.ny - 1))
                    c.pipe_nowrap = 0;
        return sync_all(c);
    }
    c.has_pipe = 1;
    c.pipe_R = radius;
    CK(launch_pipe_flags(c));
    CK(build_sites(c, 1));
    lbm_status s = sync_all(c);
    if (s != LBM_OK) return s;
    c.nsites_hint = c.nsites;
    c.nlinks_hint = c.nlinks;
    // IBB sweep work list (segments of fluid runs, see segments.h)
    std::vector<uint8_t> fl((size_t)c.N);
    CK(cudaMemcpy(fl.data(), c.flags, (size_t)c.N, cudaMemcpyDeviceToHost));
    // cells per 32-byte sector; 16-bit storage is not widened (its 16-cell
    // sectors add more zero lanes than the full-sector stores save)
    const long long sec = (LBM_SEG_SECTOR && storage_bytes(c.storage) >= 4) ? 32 / (long long)storage_bytes(c.storage) : 1;
    std::vector<unsigned long long> segs;
    const bool seg_ok = build_sweep_segments(fl.data(), c.nx, c.ny, c.nz, FL_SOLID, sec, segs);
    std::vector<SweepItem> items;
    if (seg_ok) pack_sweep_items(segs, items);
    if (seg_ok && (long long)items.size() <= c.max_seg) {
        static_assert(sizeof(SweepItem) == sizeof(uint4), "warp item layout");
        CK(cudaMemcpy(c.seg, items.data(), sizeof(SweepItem) * items.size(), cudaMemcpyHostToDevice));
        c.nseg = (long long)items.size();
    }
    // single-node links of the wall (their correction runs as its own pass)
    c.static_single = 0;
    if (c.nlinks > 0 && c.nlinks <= c.max_links) {
        std::vector<int8_t> sch((size_t)c.nlinks);
        CK(cudaMemcpy(sch.data(), c.link_scheme, (size_t)c.nlinks, cudaMemcpyDeviceToHost));
        for (int8_t v : sch) c.static_single += v == 2;
    }
    // the lean sweep needs every fluid cell off the x and y faces (no x/y wrap of a pull)
    c.pipe_nowrap = 1;
    for (long long cell = 0; cell < c.N && c.pipe_nowrap; cell++) {
        if (fl[(size_t)cell] & FL_SOLID) continue;
        const long long x = cell % c.nx, y = (cell / c.nx) % c.ny;
        if (x == 0 || x == c.nx - 1 || y == 0 || y == c.ny - 1) c.pipe_nowrap = 0;
    }
    // the wall is static: regroup its links by direction (cell order kept
    // inside a group) so that neighbouring threads of the ghost pass touch
    // neighbouring cells of one population plane
    if (LBM_STATIC_LINKS && c.storage != LBM_F64 && c.nlinks > 0 && c.nlinks <= c.max_links && c.N < (1LL << 30)) {
        const size_t nl = (size_t)c.nlinks;
        std::vector<int> lcell(nl);
        std::vector<int8_t> ldir(nl), lsch(nl);
        std::vector<double> lq(nl);
        CK(cudaMemcpy(lcell.data(), c.link_cell, 4 * nl, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(ldir.data(), c.link_dir, nl, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(lsch.data(), c.link_scheme, nl, cudaMemcpyDeviceToHost));
        CK(cudaMemcpy(lq.data(), c.link_q, 8 * nl, cudaMemcpyDeviceToHost));
        int cnt[19] = {0};
        bool ok = true;
        for (size_t k = 0; k < nl; k++) {
            if (ldir[k] < 0 || ldir[k] > 18 || lsch[k] < 0 || lsch[k] > 3) ok = false;
            else cnt[ldir[k]]++;
        }
        if (ok) {
            c.slink_off[0] = 0;
            for (int l = 0; l < 19; l++) c.slink_off[l + 1] = c.slink_off[l] + cnt[l];
            int pos[19];
            for (int l = 0; l < 19; l++) pos[l] = c.slink_off[l];
            // wall cells (cells with links; the list is in cell order) and their ranks
            std::vector<int> bcells;
            bool sorted = true;
            for (size_t k = 0; k < nl; k++) {
                if (k > 0 && lcell[k] < lcell[k - 1]) sorted = false;
                if (k == 0 || lcell[k] != lcell[k - 1]) bcells.push_back(lcell[k]);
            }
            auto rank_of = [&](long long cell) -> long long {
                auto it = std::lower_bound(bcells.begin(), bcells.end(), (int)cell);
                return (it != bcells.end() && *it == (int)cell) ? (long long)(it - bcells.begin()) : -1;
            };
            std::vector<uint2> pk(nl);
            std::vector<int> rk(nl);
            for (size_t k = 0; k < nl; k++) {
                const float qf = (float)lq[k];
                unsigned qb;
                std::memcpy(&qb, &qf, 4);
                const int at = pos[ldir[k]]++;
                pk[at] = make_uint2((unsigned)lcell[k] | ((unsigned)lsch[k] << 30), qb);
                rk[at] = (int)rank_of(lcell[k]);
            }
            CK(cudaMemcpy(c.slink, pk.data(), 8 * nl, cudaMemcpyHostToDevice));
            c.static_links = 1;
            // per sweep item: rank of its first wall cell and the lanes that hold wall cells
            bool bok = LBM_WALL_VALUES && sorted && c.nseg > 0 && (long long)bcells.size() <= c.max_bvals;
            std::vector<uint2> sb(bok ? items.size() : 0);
            std::vector<int> lane_of(bok ? bcells.size() : 0, -1);  // sweep lane of each wall cell
            for (size_t it = 0; bok && it < items.size(); it++) {
                const SweepItem &w = items[it];
                const unsigned la = (w.word_a >> 16) & 0xff;
                long long base = -1;
                unsigned mask = 0;
                for (unsigned lane = 0; lane < 32 && bok; lane++) {
                    const bool pa = lane < la;
                    const unsigned wd = pa ? w.word_a : w.word_b, row = pa ? w.row_a : w.row_b;
                    const int lp = pa ? (int)lane : (int)(lane - la);
                    const int len = (int)((wd >> 16) & 0xff), lead = (int)((wd >> 24) & 15), trail = (int)(wd >> 28);
                    if (lp >= len || lp < lead || lp >= len - trail) continue;  // idle or zero lane
                    const long long cell = (long long)row * c.nx + (long long)(wd & 0xffff) - lead + lp;
                    const long long r = rank_of(cell);
                    if (r < 0) continue;
                    if (base < 0) base = r;
                    if (r != base + __builtin_popcount(mask)) bok = false;  // ranks must follow the lanes
                    mask |= 1u << lane;
                    lane_of[(size_t)r] = (int)lane;
                }
                sb[it] = make_uint2((unsigned)(base < 0 ? 0 : base), mask);
            }
            // compact ghosts: per wall cell the directions ibar = opp(l) of its
            // links and the first of its values; per link the index of its value
            std::vector<uint2> wr(bok ? bcells.size() : 0);
            std::vector<int> gx(bok ? nl : 0);
            if (bok) {
                std::vector<unsigned> dm(bcells.size(), 0u);
                for (size_t k = 0; k < nl; k++) dm[(size_t)rank_of(lcell[k])] |= 1u << (ldir[k] == 0 ? 0 : ((ldir[k] & 1) ? ldir[k] + 1 : ldir[k] - 1));
                unsigned acc = 0;
                for (size_t r = 0; r < bcells.size(); r++) {
                    wr[r] = make_uint2(acc, dm[r]);
                    acc += (unsigned)__builtin_popcount(dm[r]);
                }
                int pos2[19];
                for (int l = 0; l < 19; l++) pos2[l] = c.slink_off[l];
                for (size_t k = 0; k < nl; k++) {
                    const int l = ldir[k], i = l == 0 ? 0 : ((l & 1) ? l + 1 : l - 1);
                    const size_t r = (size_t)rank_of(lcell[k]);
                    gx[pos2[l]++] = (int)(wr[r].x + (unsigned)__builtin_popcount(dm[r] & ((1u << i) - 1u)));
                }
                if (acc != (unsigned)nl) bok = false;  // one value per link
            }
            if (bok) {
                CK(cudaMemcpy(c.wrec, wr.data(), 8 * wr.size(), cudaMemcpyHostToDevice));
                CK(cudaMemcpy(c.gidx, gx.data(), 4 * nl, cudaMemcpyHostToDevice));
                CK(cudaMemcpy(c.slink_rank, rk.data(), 4 * nl, cudaMemcpyHostToDevice));
                CK(cudaMemcpy(c.seg_bnd, sb.data(), 8 * sb.size(), cudaMemcpyHostToDevice));
                c.bvals_ready = 1;
                c.bvals_valid = 0;
                // ghost-pass records once the wall cells' values are kept:
                // upstream cell, the two interpolation weights, wall-cell rank
                // (the linear scheme: 2q, 1 - 2q on f_l(x_f), f_l(x_f - c_l)
                // for q < 1/2; 1/(2q), (2q - 1)/(2q) on f_l(x_f), f_ibar(x_f)
                // for q >= 1/2; the single-node scheme keeps 0.5 (1 - 2q))
                std::vector<uint4> r4(nl);
                // the inline wall form's weights and lanes, in the order of the compact values
                std::vector<uint2> wc(nl);
                std::vector<unsigned short> wl(nl, 0);
                bool rok = true;
                for (size_t at = 0; at < nl && rok; at++) {
                    const unsigned cell = pk[at].x & 0x3fffffffu, sch = pk[at].x >> 30;
                    float qf;
                    std::memcpy(&qf, &pk[at].y, 4);
                    int l = 0;
                    while (l < 19 && (long long)at >= c.slink_off[l + 1]) l++;
                    const long long x = cell % c.nx, y = (cell / c.nx) % c.ny, z = cell / ((long long)c.nx * c.ny);
                    const long long x1 = (x - cx(l) + c.nx) % c.nx, y1 = (y - cy(l) + c.ny) % c.ny,
                                    z1 = (z - cz(l) + c.nz) % c.nz;
                    const unsigned c1 = (unsigned)(x1 + c.nx * (y1 + (long long)c.ny * z1));
                    const double q = (double)qf;
                    float k1, k2;
                    unsigned own = 0, single = 0;
                    if (sch == 1 && q < 0.5) {
                        k1 = (float)(2.0 * q);
                        k2 = (float)(1.0 - 2.0 * q);
                    } else if (sch == 1) {
                        k1 = (float)(1.0 / (2.0 * q));
                        k2 = (float)((2.0 * q - 1.0) / (2.0 * q));
                        own = 1;
                    } else if (sch == 2) {
                        k1 = 1.0f;
                        k2 = (float)(0.5 * (1.0 - 2.0 * q));
                        single = 1;
                    } else {
                        rok = false;  // the quadratic scheme keeps the general pass
                        break;
                    }
                    unsigned b1, b2;
                    std::memcpy(&b1, &k1, 4);
                    std::memcpy(&b2, &k2, 4);
                    r4[at] = make_uint4(c1 | (own << 30) | (single << 31), b1, b2, (unsigned)rk[at]);
                    wc[(size_t)gx[at]] = make_uint2(b1, b2 | (own << 31));
                }
                for (size_t r = 0; r < bcells.size() && rok; r++) {
                    if (lane_of[r] < 0) {
                        rok = false;  // a wall cell no sweep lane holds
                        break;
                    }
                    for (int i = 0; i < 19; i++)
                        if ((wr[r].y >> i) & 1u)
                            wl[wr[r].x + (unsigned)__builtin_popcount(wr[r].y & ((1u << i) - 1u))] =
                                (unsigned short)(lane_of[r] | (i << 5));
                }
                rok = rok && c.pipe_nowrap;  // the pass recovers x_f from x_f - c_l across z ends only
                if (rok) {
                    CK(cudaMemcpy(c.slink4, r4.data(), 16 * nl, cudaMemcpyHostToDevice));
                    CK(cudaMemcpy(c.wcoef, wc.data(), 8 * nl, cudaMemcpyHostToDevice));
                    CK(cudaMemcpy(c.wlane, wl.data(), 2 * nl, cudaMemcpyHostToDevice));
                }
                c.slink4_ready = rok ? 1 : 0;
                c.wcoef_ready = rok ? 1 : 0;
                // 16-bit storage: the pair sweep's work list and wall tables
                if (rok && (c.storage == LBM_F16S || c.storage == LBM_BF16S)) build_pair16(c, fl.data(), bcells, wr);
            }
        }
    }
    return LBM_OK;
}

lbm_status lbm_add_spheres(lbm_ctx *h, int n, const double *xyz, const double *radius, double density_ratio,
                           const double *vel, const double *omega, int fixed) {
    CTX_CHECK(h);
    if (c.q != 19) return fail(c, LBM_EUNSUPPORTED, "walls need the D3Q19 lattice");
    if (c.broken || c.armed_bc >= 0 || c.np > 0 || c.has_pipe) return fail(c, LBM_ESTATE, "geometry already set");
    if (n <= 0 || !xyz || !radius || !(density_ratio > 0)) return fail(c, LBM_EINVAL, "bad sphere arguments");
    if (n > c.max_np) return fail(c, LBM_ENOMEM, "%d spheres exceed max_particles %d", n, c.max_np);
    std::vector<double> X(xyz, xyz + 3 * n), R(radius, radius + n), m(n), I(n), zero(3 * n, 0.0);
    for (int p = 0; p < n; p++) {
        if (!(R[p] > 0.5) || !(2 * R[p] + 4 < c.nx && 2 * R[p] + 4 < c.ny && 2 * R[p] + 4 < c.nz))
            return fail(c, LBM_EINVAL, "sphere %d radius out of range", p);
        const int nn[3] = {c.nx, c.ny, c.nz};
        for (int d = 0; d < 3; d++) {
            double x = X[3 * p + d];
            if (!(x >= 0.0 && x < nn[d])) return fail(c, LBM_EINVAL, "sphere %d centre outside the box", p);
        }
        m[p] = density_ratio * 4.0 / 3.0 * M_PI * R[p] * R[p] * R[p];
        I[p] = 0.4 * m[p] * R[p] * R[p];
    }
    c.np = n;
    c.max_radius = 0.0;
    for (int p = 0; p < n; p++) c.max_radius = R[p] > c.max_radius ? R[p] : c.max_radius;
    c.fixed = fixed != 0;
    c.dens = density_ratio;
    const size_t b3 = sizeof(double) * 3 * n, b1 = sizeof(double) * n;
    CK(cudaMemcpyAsync(c.X, X.data(), b3, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(c.Xold, X.data(), b3, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(c.R, R.data(), b1, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(c.mass, m.data(), b1, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemcpyAsync(c.inertia, I.data(), b1, cudaMemcpyHostToDevice, c.stream));
    for (double *p : {c.Fh, c.Th, c.Fprev, c.Tprev, c.Iu, c.Ir})
        CK(cudaMemcpyAsync(p, zero.data(), b3, cudaMemcpyHostToDevice, c.stream));
    CK(cudaMemsetAsync(c.Fc, 0, 2 * b3, c.stream));
    CK(cudaMemsetAsync(c.has_prev, 0, sizeof(int) * n, c.stream));
    CK(cudaMemcpyAsync(c.W, omega ? omega : zero.data(), b3, cudaMemcpyHostToDevice, c.stream));
    if (vel) CK(cudaMemcpyAsync(c.U, vel, b3, cudaMemcpyHostToDevice, c.stream));
    else CK(launch_release(c));  // before the geometry exists: every cell counts as fluid
    CK(launch_sphere_mark(c, false));
    CK(build_sites(c, 1));
    lbm_status s = sync_all(c);
    if (s != LBM_OK) return s;
    c.nsites_hint = c.nsites;
    // links move with the particles: size launches with headroom
    c.nlinks_hint = c.nlinks + c.nlinks / 4 + 1024;
    return LBM_OK;
}

lbm_status lbm_step(lbm_ctx *h, int nsteps, int bc) {
    CTX_CHECK(h);
    if (nsteps < 0 || bc < LBM_BC_NONE || bc > LBM_BC_IBM_B) return fail(c, LBM_EINVAL, "bad step arguments");
    lbm_status s = check_status(c, false);
    if (s != LBM_OK) return s;
    if (c.broken) return fail(c, LBM_ESTATE, "context unusable after an error");
    // refused before the treatment is fixed, so a refused call changes nothing
    if (c.q == 27 && !(bc == LBM_BC_NONE || (bc == LBM_BC_IBB && c.has_pipe)))
        return fail(c, LBM_EUNSUPPORTED, "D3Q27 runs the periodic box and the pipe with IBB only");
    if (c.armed_bc < 0) {
        s = arm(c, bc);
        if (s != LBM_OK) return s;
    } else if (c.armed_bc != bc) {
        return fail(c, LBM_ESTATE, "boundary treatment fixed to %d by the first step", c.armed_bc);
    }
    // profiling: one event at each boundary between groups that launched
    // something (adjacent spans share it; a group that launched nothing in
    // a step records no span), so the steady pipe step carries one event
    cudaEvent_t t0 = nsteps > 0 ? pmark(c) : nullptr;
    auto close = [&](int g, long long before) {
        if (c.group_launches[g] == before) return;
        cudaEvent_t t1 = pmark(c);
        pspan(c, g, t0, t1);
        t0 = t1;
    };
    if (c.q == 27) {  // periodic box, or the pipe with its wall inside the sweep (checked above)
        for (int n = 0; n < nsteps; n++) {
            const long long b0 = c.group_launches[G_BULK];
            CK(launch_q27_step(c));
            close(G_BULK, b0);
            std::swap(c.fA, c.fB);
            c.step++;
        }
        return enqueue_status(c);
    }
    const bool ibm = bc == LBM_BC_IBM_U || bc == LBM_BC_IBM_B;
    const bool moving = c.np > 0 && !c.fixed;
    for (int n = 0; n < nsteps; n++) {
        long long b0 = c.group_launches[G_BULK];
        if (bc == LBM_BC_NONE) {
            CK(launch_stream_collide(c, bc));
            close(G_BULK, b0);
        } else if (bc == LBM_BC_IBB) {
            const long long l0 = c.group_launches[G_BND];
            CK(launch_ibb_links(c));
            close(G_BND, l0);
            b0 = c.group_launches[G_BULK];
            CK(launch_stream_collide(c, bc));
            // what the sweep left for the next step's wall
            c.bvals_valid = pipe_inline_walls(c) ? 2 : (c.bvals_ready ? 1 : 0);
            close(G_BULK, b0);
            const long long p0 = c.group_launches[G_PART];
            if (c.np > 0) CK(launch_gimem(c));
            if (moving) CK(launch_particle_update(c));
            close(G_PART, p0);
            const long long g0 = c.group_launches[G_GEOM];
            if (moving) {
                CK(launch_sphere_mark(c, true));
                CK(launch_refill(c));
                CK(launch_finish_geometry(c));
                CK(build_sites(c, 1));
            }
            close(G_GEOM, g0);
        } else if (ibm) {
            long long g0 = c.group_launches[G_GEOM];
            if (moving && c.step > 0) {
                CK(launch_support_mark(c));
                CK(build_sites(c, 2));
            }
            close(G_GEOM, g0);
            b0 = c.group_launches[G_BULK];
            CK(launch_stream_collide(c, bc));
            close(G_BULK, b0);
            const long long i0 = c.group_launches[G_IBM];
            CK(launch_ibm_passes(c));
            close(G_IBM, i0);
            const long long k0 = c.group_launches[G_IBMCOL];
            CK(launch_ibm_collide(c));
            close(G_IBMCOL, k0);
            const long long p0 = c.group_launches[G_PART];
            if (c.np > 0) CK(launch_ibm_particle_sums(c, false));
            if (moving) CK(launch_particle_update(c));
            close(G_PART, p0);
            g0 = c.group_launches[G_GEOM];
            if (moving) {
                CK(launch_markers_place(c));
                CK(launch_marker_offsets(c));
                CK(launch_sphere_mark(c, true));
                CK(launch_finish_geometry(c));
            }
            close(G_GEOM, g0);
        }
        std::swap(c.fA, c.fB);
        c.step++;
    }
    return enqueue_status(c);
}

lbm_status lbm_stats(lbm_ctx *h, int flags, lbm_stats_t *out) {
    CTX_CHECK(h);
    if (!out) return fail(c, LBM_EINVAL, "null output");
    lbm_status s = sync_all(c);
    if (s != LBM_OK && s != LBM_EUNSTABLE) return s;
    CK(run_stats(c, flags, out));
    out->nlinks = c.nlinks;
    return s;
}

lbm_status lbm_spectrum(lbm_ctx *h, int flags, int nbins, double *E, double *D) {
    CTX_CHECK(h);
    if (!E || !D || nbins < 1 || nbins > LBM_SPECTRUM_MAX_BINS) return fail(c, LBM_EINVAL, "bad spectrum arguments");
    const int n = c.nx;
    if (c.ny != n || c.nz != n || n < 8 || n > 1024 || (n & (n - 1)) != 0)
        return fail(c, LBM_EUNSUPPORTED, "spectra need a cube of side 2^k, 8 <= side <= 1024 (grid %dx%dx%d)", c.nx,
                    c.ny, c.nz);
    if (spectrum_scratch_bytes(c.N, nbins) > 19 * (size_t)c.N * storage_bytes(c.storage))
        return fail(c, LBM_ENOMEM, "spectrum scratch does not fit the idle population buffer");
    lbm_status s = sync_all(c);
    if (s != LBM_OK && s != LBM_EUNSTABLE) return s;
    CK(run_spectrum(c, flags, nbins, E, D));
    return s;
}

lbm_status lbm_pipe_profiles(lbm_ctx *h, int flags, int nbins, double *out) {
    CTX_CHECK(h);
    if (!out || nbins < 1 || nbins > LBM_PROF_MAX_BINS) return fail(c, LBM_EINVAL, "bad profile arguments");
    if (!c.has_pipe) return fail(c, LBM_ESTATE, "no pipe");
    if (pipe_profile_scratch_bytes(nbins) > 19 * (size_t)c.N * storage_bytes(c.storage))
        return fail(c, LBM_ENOMEM, "profile scratch does not fit the idle population buffer");
    lbm_status s = sync_all(c);
    if (s != LBM_OK && s != LBM_EUNSTABLE) return s;
    CK(run_pipe_profiles(c, flags, nbins, out));
    return s;
}

lbm_status lbm_set_mrt_rates(lbm_ctx *h, double s_e, double s_eps, double s_q, double s_pi, double s_m) {
    CTX_CHECK(h);
    if (c.q != 19) return fail(c, LBM_EUNSUPPORTED, "the MRT collision is built for D3Q19");
    const double v[5] = {s_e, s_eps, s_q, s_pi, s_m};
    for (double x : v)
        if (!(x > 0.0 && x < 2.0)) return fail(c, LBM_EINVAL, "relaxation rates must lie in (0, 2)");
    // kernels take the rates by value at launch: the change applies from the next step
    c.rates = LBM_RATES_DHUMIERES;
    Rates &r = c.rt;
    r.d_e = s_e;
    r.d_eps = s_eps;
    r.d_q = s_q;
    r.d_pi = s_pi;
    r.d_m = s_m;
    r.s_e = (float)s_e;
    r.s_eps = (float)s_eps;
    r.s_q = (float)s_q;
    r.s_pi = (float)s_pi;
    r.s_m = (float)s_m;
    return LBM_OK;
}

lbm_status lbm_tke_budget(lbm_ctx *h, int flags, int nbins, double *out) {
    CTX_CHECK(h);
    if (!out || nbins < 1 || nbins > LBM_PROF_MAX_BINS) return fail(c, LBM_EINVAL, "bad budget arguments");
    if (!c.has_pipe) return fail(c, LBM_ESTATE, "no pipe");
    if (tke_budget_scratch_bytes(nbins) > 19 * (size_t)c.N * storage_bytes(c.storage))
        return fail(c, LBM_ENOMEM, "budget scratch does not fit the idle population buffer");
    lbm_status s = sync_all(c);
    if (s != LBM_OK && s != LBM_EUNSTABLE) return s;
    CK(run_tke_budget(c, flags, nbins, out));
    return s;
}

lbm_status lbm_get_field(lbm_ctx *h, int which, void *dst, size_t bytes) {
    CTX_CHECK(h);
    if (!dst) return fail(c, LBM_EINVAL, "null destination");
    lbm_status s = sync_all(c);
    if (s != LBM_OK && s != LBM_EUNSTABLE) return s;
    const size_t N = (size_t)c.N;
    switch (which) {
    case LBM_FIELD_RHO:
    case LBM_FIELD_U: {
        const size_t need = (which == LBM_FIELD_RHO ? 1 : 3) * N * sizeof(double);
        if (bytes < need) return fail(c, LBM_EINVAL, "destination too small");
        CK(launch_macro(c, 0));
        CK(cudaMemcpyAsync(dst, which == LBM_FIELD_RHO ? (void *)c.rho_f : (void *)c.u_f, need,
                           cudaMemcpyDeviceToHost, c.stream));
        break;
    }
    case LBM_FIELD_POPS: {
        if (bytes < (size_t)c.q * N * sizeof(double)) return fail(c, LBM_EINVAL, "destination too small");
        for (int i = 0; i < c.q; i++) {
            if (c.q == 27) CK(q27_plane_copy(c, i, true));
            else CK(plane_copy(c, i, true));
            CK(cudaMemcpyAsync((double *)dst + i * N, c.rho_f, N * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        }
        break;
    }
    case LBM_FIELD_FLAGS: {
        if (bytes < N) return fail(c, LBM_EINVAL, "destination too small");
        CK(cudaMemcpyAsync(dst, c.flags, N, cudaMemcpyDeviceToHost, c.stream));
        CK(cudaStreamSynchronize(c.stream));
        uint8_t *f = (uint8_t *)dst;
        for (size_t i = 0; i < N; i++) f[i] &= (FL_SOLID | FL_BND | FL_SUP);
        break;
    }
    case LBM_FIELD_IBM_FORCE: {
        if (bytes < 3 * N * sizeof(double)) return fail(c, LBM_EINVAL, "destination too small");
        CK(cudaMemsetAsync(c.u_f, 0, 3 * N * sizeof(double), c.stream));
        if (c.armed_bc == LBM_BC_IBM_U || c.armed_bc == LBM_BC_IBM_B)
        {
            if (c.storage == LBM_F64)
                dense_ibm_force<double><<<1024, 256, 0, c.stream>>>(c.u_f, (const double *)c.sup_F, c.site_cell,
                                                                     c.d_counts, c.max_sites, c.N);
            else
                dense_ibm_force<float><<<1024, 256, 0, c.stream>>>(c.u_f, (const float *)c.sup_F, c.site_cell,
                                                                    c.d_counts, c.max_sites, c.N);
        }
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(dst, c.u_f, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        break;
    }
    default:
        return fail(c, LBM_EINVAL, "unknown field %d", which);
    }
    CK(cudaStreamSynchronize(c.stream));
    return s;
}

lbm_status lbm_num_links(lbm_ctx *h, long long *n) {
    CTX_CHECK(h);
    if (!n) return LBM_EINVAL;
    lbm_status s = sync_all(c);
    *n = c.nlinks;
    return s;
}

lbm_status lbm_get_links(lbm_ctx *h, long long capacity, long long *cell, int *dir, int *scheme, double *q, int *pid) {
    CTX_CHECK(h);
    lbm_status s = sync_all(c);
    if (s != LBM_OK && s != LBM_EUNSTABLE) return s;
    const long long n = c.nlinks < c.max_links ? c.nlinks : c.max_links;
    if (capacity < n) return fail(c, LBM_EINVAL, "capacity %lld < %lld links", capacity, n);
    if (n == 0) return s;
    std::vector<int> ic(n), ip(n);
    std::vector<int8_t> id(n), is(n);
    CK(cudaMemcpyAsync(ic.data(), c.link_cell, 4 * n, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(ip.data(), c.link_pid, 4 * n, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(id.data(), c.link_dir, n, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaMemcpyAsync(is.data(), c.link_scheme, n, cudaMemcpyDeviceToHost, c.stream));
    if (q) CK(cudaMemcpyAsync(q, c.link_q, 8 * n, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    for (long long k = 0; k < n; k++) {
        if (cell) cell[k] = ic[k];
        if (dir) dir[k] = id[k];
        if (scheme) scheme[k] = is[k];
        if (pid) pid[k] = ip[k];
    }
    return s;
}

lbm_status lbm_get_particles(lbm_ctx *h, double *X, double *U, double *W, double *F, double *T) {
    CTX_CHECK(h);
    lbm_status s = sync_all(c);
    if (s != LBM_OK && s != LBM_EUNSTABLE) return s;
    const size_t b3 = sizeof(double) * 3 * c.np;
    if (c.np == 0) return s;
    if (X) CK(cudaMemcpyAsync(X, c.X, b3, cudaMemcpyDeviceToHost, c.stream));
    if (U) CK(cudaMemcpyAsync(U, c.U, b3, cudaMemcpyDeviceToHost, c.stream));
    if (W) CK(cudaMemcpyAsync(W, c.W, b3, cudaMemcpyDeviceToHost, c.stream));
    if (F) CK(cudaMemcpyAsync(F, c.Fh, b3, cudaMemcpyDeviceToHost, c.stream));
    if (T) CK(cudaMemcpyAsync(T, c.Th, b3, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return s;
}

lbm_status lbm_num_particles(lbm_ctx *h, int *n) {
    CTX_CHECK(h);
    if (!n) return LBM_EINVAL;
    *n = c.np;
    return LBM_OK;
}

lbm_status lbm_num_markers(lbm_ctx *h, long long *n) {
    CTX_CHECK(h);
    if (!n) return LBM_EINVAL;
    *n = c.nm;
    return LBM_OK;
}

lbm_status lbm_get_markers(lbm_ctx *h, long long capacity, double *X, double *F, double *dV, int *pid) {
    CTX_CHECK(h);
    lbm_status s = sync_all(c);
    if (s != LBM_OK && s != LBM_EUNSTABLE) return s;
    if (capacity < c.nm) return fail(c, LBM_EINVAL, "capacity %lld < %lld markers", capacity, c.nm);
    if (c.nm == 0) return s;
    if (X) CK(cudaMemcpyAsync(X, c.mX, 24 * c.nm, cudaMemcpyDeviceToHost, c.stream));
    if (F) CK(cudaMemcpyAsync(F, c.mFacc, 24 * c.nm, cudaMemcpyDeviceToHost, c.stream));
    if (dV) CK(cudaMemcpyAsync(dV, c.mdV, 8 * c.nm, cudaMemcpyDeviceToHost, c.stream));
    if (pid) CK(cudaMemcpyAsync(pid, c.mpid, 4 * c.nm, cudaMemcpyDeviceToHost, c.stream));
    CK(cudaStreamSynchronize(c.stream));
    return s;
}

lbm_status lbm_set_wait_limit(lbm_ctx *h, double seconds) {
    CTX_CHECK(h);
    if (!(seconds > 0.0 && seconds <= 1e6)) return fail(c, LBM_EINVAL, "wait limit must lie in (0, 1e6] s");
    c.wait_limit_s = seconds;
    return LBM_OK;
}

}  // extern "C"

namespace lbmgb {
namespace {

// Checkpoint file: this header, then raw arrays in host byte order (see
// lbm_checkpoint in lbm.h for the list and their order).
struct CkptHeader {
    char magic[8];  // "LBMCKPT\0"
    int version, nx, ny, nz, storage, q, rates, armed_bc, has_pipe, np, fixed, cl_ready;
    double tau, F[3], rt[6];  // rates: e, eps, q, nu, pi, m
    double pipe_R, dens, cl_uscale, cl_gscale;
    long long step, nsites, nm;
};
constexpr int CKPT_VERSION = 1;
constexpr size_t CKPT_CHUNK = 64u << 20;  // bytes staged through host memory at a time

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

lbm_status io_fail(Ctx &c, const char *what, const char *path) {
    return fail(c, LBM_EIO, "checkpoint %s failed: %s", what, path);
}

// device -> file and file -> device through a bounded host buffer
lbm_status dev_to_file(Ctx &c, FILE *f, const void *dev, size_t bytes, const char *path) {
    std::vector<char> buf(std::min(bytes, CKPT_CHUNK));
    for (size_t o = 0; o < bytes; o += CKPT_CHUNK) {
        const size_t n = std::min(CKPT_CHUNK, bytes - o);
        CK(cudaMemcpyAsync(buf.data(), (const char *)dev + o, n, cudaMemcpyDeviceToHost, c.stream));
        CK(cudaStreamSynchronize(c.stream));
        if (fwrite(buf.data(), 1, n, f) != n) return io_fail(c, "write", path);
    }
    return LBM_OK;
}
lbm_status file_to_dev(Ctx &c, FILE *f, void *dev, size_t bytes, const char *path) {
    std::vector<char> buf(std::min(bytes, CKPT_CHUNK));
    for (size_t o = 0; o < bytes; o += CKPT_CHUNK) {
        const size_t n = std::min(CKPT_CHUNK, bytes - o);
        if (fread(buf.data(), 1, n, f) != n) return io_fail(c, "read (truncated file)", path);
        CK(cudaMemcpyAsync((char *)dev + o, buf.data(), n, cudaMemcpyHostToDevice, c.stream));
        CK(cudaStreamSynchronize(c.stream));
    }
    return LBM_OK;
}

#define CKS(call)                                  \
    do {                                           \
        lbm_status s_ = (call);                    \
        if (s_ != LBM_OK) return s_;               \
    } while (0)

size_t arith_bytes(const Ctx &c) { return c.storage == LBM_F64 ? 8 : 4; }

// support set of the last IBM step (a moving particle's set is rebuilt at
// the start of the next step): clear the support flags, then mark the listed cells
__global__ void clear_support_kernel(uint8_t *flags, long long N) {
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c < N) flags[c] = (uint8_t)(flags[c] & ~FL_SUP);
}
__global__ void mark_support_kernel(uint8_t *flags, const int *cells, long long n) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) flags[cells[k]] = (uint8_t)(flags[cells[k]] | FL_SUP);
}

}  // namespace
}  // namespace lbmgb

extern "C" {

lbm_status lbm_checkpoint(lbm_ctx *h, const char *path) {
    CTX_CHECK(h);
    if (!path) return fail(c, LBM_EINVAL, "null path");
    if (c.broken) return fail(c, LBM_ESTATE, "context unusable after an error");
    lbm_status s = sync_all(c);
    if (s != LBM_OK) return s;
    CkptHeader H;
    memset(&H, 0, sizeof(H));
    memcpy(H.magic, "LBMCKPT", 8);
    H.version = CKPT_VERSION;
    H.nx = c.nx;
    H.ny = c.ny;
    H.nz = c.nz;
    H.storage = c.storage;
    H.q = c.q;
    H.rates = c.rates;
    H.armed_bc = c.armed_bc;
    H.has_pipe = c.has_pipe;
    H.np = c.np;
    H.fixed = c.fixed;
    H.cl_ready = c.cl_ready;
    H.tau = c.tau;
    for (int d = 0; d < 3; d++) H.F[d] = c.F[d];
    const double rt[6] = {c.rt.d_e, c.rt.d_eps, c.rt.d_q, c.rt.d_nu, c.rt.d_pi, c.rt.d_m};
    for (int k = 0; k < 6; k++) H.rt[k] = rt[k];
    H.pipe_R = c.pipe_R;
    H.dens = c.dens;
    H.cl_uscale = c.cl_uscale;
    H.cl_gscale = c.cl_gscale;
    H.step = c.step;
    const bool ibm = c.armed_bc == LBM_BC_IBM_U || c.armed_bc == LBM_BC_IBM_B;
    H.nsites = ibm ? c.nsites : 0;
    H.nm = ibm ? c.nm : 0;
    File F;
    F.f = fopen(path, "wb");
    if (!F.f) return io_fail(c, "open", path);
    if (fwrite(&H, sizeof(H), 1, F.f) != 1) return io_fail(c, "write", path);
    CKS(dev_to_file(c, F.f, c.fA, (size_t)c.q * (size_t)c.N * storage_bytes(c.storage), path));
    if (c.np > 0) {
        const size_t b3 = sizeof(double) * 3 * (size_t)c.np;
        for (const double *p : {c.X, c.U, c.W, c.Fh, c.Th, c.Fprev, c.Tprev, c.Fc, c.Iu, c.Ir})
            CKS(dev_to_file(c, F.f, p, b3, path));
        CKS(dev_to_file(c, F.f, c.R, sizeof(double) * (size_t)c.np, path));
        CKS(dev_to_file(c, F.f, c.has_prev, sizeof(int) * (size_t)c.np, path));
    }
    if (H.nsites > 0) {
        CKS(dev_to_file(c, F.f, c.site_cell, sizeof(int) * (size_t)H.nsites, path));
        CKS(dev_to_file(c, F.f, c.sup_F, 3 * arith_bytes(c) * (size_t)H.nsites, path));
    }
    if (H.nm > 0) CKS(dev_to_file(c, F.f, c.mFacc, sizeof(double) * 3 * (size_t)H.nm, path));
    if (c.cl_ready) CKS(dev_to_file(c, F.f, c.cl_w, sizeof(float) * LBM_MLP_NPARAM, path));
    if (fflush(F.f) != 0) return io_fail(c, "write", path);
    return LBM_OK;
}

lbm_status lbm_restore(lbm_ctx *h, const char *path) {
    CTX_CHECK(h);
    if (!path) return fail(c, LBM_EINVAL, "null path");
    if (c.broken || c.armed_bc >= 0 || c.np > 0 || c.has_pipe || c.step != 0)
        return fail(c, LBM_ESTATE, "restore needs a freshly created context");
    File F;
    F.f = fopen(path, "rb");
    if (!F.f) return io_fail(c, "open", path);
    CkptHeader H;
    if (fread(&H, sizeof(H), 1, F.f) != 1 || memcmp(H.magic, "LBMCKPT", 8) != 0 || H.version != CKPT_VERSION)
        return io_fail(c, "read (not a checkpoint of this version)", path);
    if (H.nx != c.nx || H.ny != c.ny || H.nz != c.nz || H.storage != c.storage || H.q != c.q || H.tau != c.tau ||
        H.F[0] != c.F[0] || H.F[1] != c.F[1] || H.F[2] != c.F[2])
        return fail(c, LBM_EINVAL, "checkpoint of another grid, storage, lattice, tau or force");
    if (H.np < 0 || H.np > c.max_np) return fail(c, LBM_ENOMEM, "%d particles exceed max_particles %d", H.np, c.max_np);
    if (H.armed_bc < -1 || H.armed_bc > LBM_BC_IBM_B || H.nsites < 0 || H.nm < 0 || H.step < 0)
        return io_fail(c, "read (corrupt header)", path);
    // relaxation rates (lbm_set_mrt_rates may have changed them)
    c.rates = H.rates;
    Rates &r = c.rt;
    r.d_e = H.rt[0];
    r.d_eps = H.rt[1];
    r.d_q = H.rt[2];
    r.d_nu = H.rt[3];
    r.d_pi = H.rt[4];
    r.d_m = H.rt[5];
    r.s_e = (float)r.d_e;
    r.s_eps = (float)r.d_eps;
    r.s_q = (float)r.d_q;
    r.s_nu = (float)r.d_nu;
    r.s_pi = (float)r.d_pi;
    r.s_m = (float)r.d_m;
    const size_t pop_bytes = (size_t)c.q * (size_t)c.N * storage_bytes(c.storage);
    // the populations come first in the file: skip them to rebuild the geometry
    if (fseek(F.f, (long)pop_bytes, SEEK_CUR) != 0) return io_fail(c, "seek", path);
    std::vector<double> P3[10], R;
    std::vector<int> has;
    if (H.np > 0) {
        for (auto &v : P3) {
            v.resize(3 * (size_t)H.np);
            if (fread(v.data(), sizeof(double), v.size(), F.f) != v.size()) return io_fail(c, "read", path);
        }
        R.resize((size_t)H.np);
        has.resize((size_t)H.np);
        if (fread(R.data(), sizeof(double), R.size(), F.f) != R.size()) return io_fail(c, "read", path);
        if (fread(has.data(), sizeof(int), has.size(), F.f) != has.size()) return io_fail(c, "read", path);
    }
    // geometry and wall treatment, rebuilt from the saved positions exactly as the first set-up built them
    if (H.has_pipe) CKS(lbm_set_pipe(h, H.pipe_R));
    if (H.np > 0)
        CKS(lbm_add_spheres(h, H.np, P3[0].data(), R.data(), H.dens, P3[1].data(), P3[2].data(), H.fixed));
    if (H.armed_bc >= 0) CKS(arm(c, H.armed_bc));
    // then the saved state over what the set-up computed
    if (fseek(F.f, (long)sizeof(H), SEEK_SET) != 0) return io_fail(c, "seek", path);
    CKS(file_to_dev(c, F.f, c.fA, pop_bytes, path));
    c.bvals_valid = 0;  // the next ghost pass reads the wall cells from the populations
    if (H.np > 0) {
        if (fseek(F.f, (long)(sizeof(double) * (10 * 3 + 1) * (size_t)H.np + sizeof(int) * (size_t)H.np), SEEK_CUR) != 0)
            return io_fail(c, "seek", path);
        const size_t b3 = sizeof(double) * 3 * (size_t)H.np;
        double *dst[10] = {c.X, c.U, c.W, c.Fh, c.Th, c.Fprev, c.Tprev, c.Fc, c.Iu, c.Ir};
        for (int k = 0; k < 10; k++) CK(cudaMemcpyAsync(dst[k], P3[k].data(), b3, cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemcpyAsync(c.Xold, P3[0].data(), b3, cudaMemcpyHostToDevice, c.stream));
        CK(cudaMemcpyAsync(c.has_prev, has.data(), sizeof(int) * has.size(), cudaMemcpyHostToDevice, c.stream));
        CK(cudaStreamSynchronize(c.stream));
    }
    if (H.nsites > 0) {
        // the support set of the last step (moving particles: the positions
        // before their last update), whose IBM force the statistics use
        if (H.nsites > c.max_sites || (size_t)H.nsites * sizeof(int) > 24 * (size_t)c.N)
            return fail(c, LBM_ENOMEM, "checkpoint support set exceeds max_sites");
        int *cells = (int *)c.u_f;  // statistics scratch as staging
        CKS(file_to_dev(c, F.f, cells, sizeof(int) * (size_t)H.nsites, path));
        clear_support_kernel<<<(unsigned)((c.N + 255) / 256), 256, 0, c.stream>>>(c.flags, c.N);
        mark_support_kernel<<<(unsigned)((H.nsites + 255) / 256), 256, 0, c.stream>>>(c.flags, cells, H.nsites);
        CK(cudaGetLastError());
        CK(build_sites(c, 2));
        CKS(sync_all(c));
        if (H.nsites != c.nsites) return fail(c, LBM_EINVAL, "checkpoint support set is not a support set of this grid");
        c.nsites_hint = c.nsites;
        CKS(file_to_dev(c, F.f, c.sup_F, 3 * arith_bytes(c) * (size_t)H.nsites, path));
    }
    if (H.nm > 0) {
        if (H.nm != c.nm) return fail(c, LBM_EINVAL, "checkpoint markers differ from the rebuilt ones");
        CKS(file_to_dev(c, F.f, c.mFacc, sizeof(double) * 3 * (size_t)H.nm, path));
    }
    if (H.cl_ready) {
        if (c.max_cl == 0) return fail(c, LBM_EUNSUPPORTED, "closure weights need max_particles > 0");
        CKS(file_to_dev(c, F.f, c.cl_w, sizeof(float) * LBM_MLP_NPARAM, path));
        c.cl_uscale = H.cl_uscale;
        c.cl_gscale = H.cl_gscale;
        c.cl_ready = 1;
    }
    c.step = H.step;
    return sync_all(c);
}

lbm_status lbm_closure_set_weights(lbm_ctx *h, const float *w_host, int n, double u_scale, double g_scale) {
    CTX_CHECK(h);
    if (!w_host || n != 14409 || !(u_scale > 0) || !(g_scale > 0)) return fail(c, LBM_EINVAL, "bad closure weights");
    if (c.max_cl == 0) return fail(c, LBM_EUNSUPPORTED, "closure needs max_particles > 0");
    CK(cudaMemcpy(c.cl_w, w_host, sizeof(float) * n, cudaMemcpyHostToDevice));
    c.cl_uscale = u_scale;
    c.cl_gscale = g_scale;
    c.cl_ready = 1;
    return LBM_OK;
}

lbm_status lbm_closure_samples(lbm_ctx *h, double u_scale, float *X_dev, int *cells_dev, long long capacity,
                               long long *n) {
    CTX_CHECK(h);
    if (!X_dev || !cells_dev || !n || capacity < 0 || !(u_scale > 0)) return fail(c, LBM_EINVAL, "bad arguments");
    if (c.np == 0) return fail(c, LBM_ESTATE, "no particles");
    lbm_status s = sync_all(c);
    if (s != LBM_OK) return s;
    CK(closure_samples(c, u_scale, X_dev, cells_dev, capacity, n));
    if (*n > capacity) return fail(c, LBM_ENOMEM, "%lld near-surface nodes exceed capacity %lld", *n, capacity);
    return LBM_OK;
}

lbm_status lbm_closure_targets(lbm_ctx *h, const int *cells_dev, long long n, double g_scale, float *T_dev) {
    CTX_CHECK(h);
    if ((n > 0 && (!cells_dev || !T_dev)) || n < 0 || !(g_scale > 0)) return fail(c, LBM_EINVAL, "bad arguments");
    lbm_status s = sync_all(c);
    if (s != LBM_OK) return s;
    CK(closure_targets(c, cells_dev, n, g_scale, T_dev));
    CK(cudaStreamSynchronize(c.stream));
    return LBM_OK;
}

lbm_status lbm_profile(lbm_ctx *h, int enable, lbm_profile_t *out) {
    CTX_CHECK(h);
    if (!c.prof) c.prof = new Prof();
    Prof *P = (Prof *)c.prof;
    if (out) {
        CK(cudaStreamSynchronize(c.stream));
        // adjacent spans share their boundary event: return each event once
        std::vector<cudaEvent_t> used;
        for (auto &r : P->recs) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) {
                P->ms[r.group] += ms;
                P->spans[r.group]++;
            }
            used.push_back(r.a);
            used.push_back(r.b);
        }
        P->recs.clear();
        std::sort(used.begin(), used.end());
        used.erase(std::unique(used.begin(), used.end()), used.end());
        P->pool.insert(P->pool.end(), used.begin(), used.end());
        memset(out, 0, sizeof(*out));
        for (int g = 0; g < LBM_NGROUPS; g++) {
            out->ms[g] = P->ms[g];
            out->spans[g] = P->spans[g];
            out->launches[g] = c.group_launches[g] - P->launches0[g];
        }
        out->total_launches = c.launches;
    }
    if (enable >= 0) {
        const int was = c.prof_on;
        c.prof_on = enable ? 1 : 0;
        if (enable && !was) {
            for (int g = 0; g < LBM_NGROUPS; g++) {
                P->ms[g] = 0.0;
                P->spans[g] = 0;
                P->launches0[g] = c.group_launches[g];
            }
        }
    }
    return LBM_OK;
}

const char *lbm_last_error(const lbm_ctx *h) { return h ? h->c.err : "null context"; }

const char *lbm_status_string(int s) {
    switch (s) {
    case LBM_OK: return "ok";
    case LBM_EINVAL: return "invalid argument";
    case LBM_ENOMEM: return "workspace or capacity too small";
    case LBM_ECUDA: return "CUDA error";
    case LBM_EUNSTABLE: return "numerical instability detected";
    case LBM_ETIMEOUT: return "timed out waiting for the GPU";
    case LBM_ESTATE: return "call not allowed in this state";
    case LBM_EUNSUPPORTED: return "unsupported";
    case LBM_EIO: return "checkpoint file error";
    default: return "unknown status";
    }
}

void lbm_destroy(lbm_ctx *h) {
    if (!h) return;
    Ctx &c = h->c;
    cudaStreamSynchronize(c.stream);
    if (c.prof) {
        Prof *P = (Prof *)c.prof;
        std::vector<cudaEvent_t> all(P->pool);
        for (auto &r : P->recs) {
            all.push_back(r.a);
            all.push_back(r.b);
        }
        std::sort(all.begin(), all.end());
        all.erase(std::unique(all.begin(), all.end()), all.end());
        for (auto e : all) cudaEventDestroy(e);
        delete P;
    }
    if (c.ev_status) cudaEventDestroy(c.ev_status);
    if (c.h_status) cudaFreeHost(c.h_status);
    delete h;
}

}  // extern "C"
