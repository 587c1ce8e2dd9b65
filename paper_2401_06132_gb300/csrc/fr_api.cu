// fr_api.cu -- mesh set-up and the C ABI of the GB300 flux-reconstruction library.
#include <cuda_runtime.h>

#include <cmath>
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "fr_internal.h"

// ---------------------------------------------------------------------------------------------
// Errors
// ---------------------------------------------------------------------------------------------
static thread_local std::string g_err;

static fr_status fail(fr_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

#define CU(call)                                                                               \
    do {                                                                                       \
        cudaError_t _e = (call);                                                               \
        if (_e != cudaSuccess) return fail(FR_ECUDA, "%s: %s", #call, cudaGetErrorString(_e)); \
    } while (0)

extern "C" const char *fr_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------------------------
// Handle
// ---------------------------------------------------------------------------------------------
struct InstanceHost {
    fr_params prm;
    int n_hex, n_pri, n_tet, n_pyr;
    std::vector<double> x0J;   // per element: x0[3], J[9] (row-major dx_i/dxi_j); x = x0 + J (xi + 1)
    std::vector<char> curved;  // per element: 1 = non-affine (trilinear) hexahedron
    std::vector<double> vx;    // per element: the 8 hexahedron vertices (tensor order), [24]
};

// Blocks of one element type and order, launched together (one launch per phase).
struct Group {
    int type = 0, p = 0, m = 0;
    std::vector<int> blks;
    long long ne = 0;
    void *d_geo = nullptr;          // Geo<T> per element in group order (multi-block groups)
    long long *d_eu0 = nullptr, *d_ef0 = nullptr;
    int *d_eph = nullptr;
    void *d_phtab = nullptr;        // Phys<T> per instance
    uint32_t *d_lpts = nullptr;     // L flux points of the group (element_in_group * 256 + local)
    int variant = 1;                // volume-kernel launch shape (autotuned: 0, 1, 2 = 64, 128, 256 threads)
    void *d_geo64 = nullptr;        // GeoLM per element in group order (low-Mach form)
    void *d_fnrm = nullptr;         // face normal table in group order
    double *d_fnrm64 = nullptr;
    long long nlpts = 0;
};

struct fr_mesh {
    int dev = 0;
    int nsm = 1;                         // streaming multiprocessors of the device
    // partitioned single mesh (fr_mesh_create_part): this handle owns the global elements [E0, E1)
    // of a mesh split into nparts contiguous ranges; flux points nfpt_own .. nfpt - 1 are halo slots
    // holding the face data of remote partners, peer by peer (halo_off[q] .. halo_off[q + 1] - 1)
    int nparts = 1, part = 0;
    long long E0 = 0, E1 = 0, nfpt_own = 0;
    std::vector<long long> halo_off;     // [nparts + 1] prefix sums of the points exchanged per peer
    uint32_t *d_send = nullptr;          // own flux points sent to the peers, in buffer order
    int prec = FR_FP64;
    int form = FR_FUSED;
    std::vector<InstanceHost> inst;
    std::vector<Block> blocks;
    std::vector<long long> inst_u0;      // value offsets per instance (+ total)
    long long ne = 0, nU = 0, nfpt = 0, npair = 0;
    std::vector<frb::Hex1D> hex1d;       // per block (hex; for prisms the z operators)
    frb::Prism2D pri;                    // prism operators (p = 3)
    bool has_pri = false;
    void *d_priops = nullptr;            // PriOps<T> on the device
    void *d_priops64 = nullptr;          // PriOpsFF (low-Mach FP32 form with prisms)
    frb::Tet3D tet;                      // tetrahedron operators (p = 3)
    bool has_tet = false;
    void *d_tetops = nullptr;            // TetOps<T> on the device
    void *d_tetops64 = nullptr;          // DenseOpsFF<TetOps<float>> (low-Mach FP32 form)
    frb::Pyr3D pyr;                      // pyramid operators (p = 3)
    bool has_pyr = false;
    void *d_pyrops = nullptr;            // PyrOps<T> on the device
    void *d_pyrops64 = nullptr;          // DenseOpsFF<PyrOps<float>> (low-Mach FP32 form)
    std::vector<Group> groups;
    bool split_c = false;              // interface phase as pair flux (C1) + lift (C2)
    bool lowmach = false;              // FP32 low-Mach form (deviations, reduced energy, FP64 mass)
    void *d_geo64 = nullptr;           // FP64 geometry for the low-Mach form
    double *d_MF = nullptr, *d_RL = nullptr;
    std::vector<double> fnrm_host;     // [elem][6][4] unit normal and |n_s| per face
    void *d_fnrm = nullptr;            // same in the compute precision
    double *d_fnrm64 = nullptr;        // float-float copy (low-Mach form; 8 bytes per entry)
    std::vector<double> geo_host;        // per element Ji[9], det (FP64)
    // device
    void *d_geo = nullptr;               // Geo<T>[ne]
    uint32_t *d_partner = nullptr;
    void *d_UF = nullptr, *d_FV = nullptr;
    void *d_CF = nullptr, *d_QF = nullptr, *d_DF = nullptr, *d_Qu = nullptr, *d_UQ = nullptr, *d_QQ = nullptr, *d_Rt = nullptr;
    void *d_rk_k = nullptr, *d_rk_us = nullptr;
    double *d_rk_acc = nullptr;
    void *d_io_U = nullptr, *d_io_R = nullptr;     // staging for the host-buffer variants
    void *d_Qsnap = nullptr;                       // debug: gradient snapshot of the unfused form
    int debug = 0;
    double *d_wsum = nullptr;                      // diagnostics accumulators
    double *d_wts = nullptr;                       // [elem] -> W per point handled in-kernel
    int *d_status = nullptr;
    int *h_status = nullptr;                       // pinned
    cudaEvent_t ev_status = nullptr;
    bool status_pending = false;
    long long bytes = 0;
    // optional per-kernel timing: events recorded around each launch on the launching stream
    bool timing = false;
    struct Timed { int kernel; cudaEvent_t a, b; };
    std::vector<Timed> timed;
    std::vector<cudaEvent_t> ev_pool;
    // CUDA graph of one RK4 step (captured on first use, replayed per step)
    bool use_graph = true;
    cudaGraphExec_t graph = nullptr;
    const void *graph_U = nullptr;
    double graph_dt = 0;
    cudaStream_t graph_stream = nullptr;
    int graph_form = -1;
    int hex_tc = 0;                      // mixed forms: hexahedral plane contractions on the tensor cores
    int merged = 0;                      // one launch per phase over all groups (fr_set_merged, fr_autotune)
    int rk_wide = 0;                     // reduced precisions: RK4 stage states and sum in FP64 (fr_set_rk_fp64_stages)
    int dense_tc = 0;                    // mixed forms: tetrahedral / pyramidal interpolation on the tensor cores
    // surface-flux anti-aliasing: face quadrature points (m x m per hex face) as interface points
    bool surf = false;
    long long nqf = 0;                   // face quadrature points of the handle
    std::vector<uint32_t> qpartner_host;
    uint32_t *d_qpartner = nullptr, *d_qlpts = nullptr;
    long long nqlpts = 0;
    void *d_UFQ = nullptr, *d_FVQ = nullptr, *d_DQ = nullptr;
    // curved (trilinear) hexahedra: metric terms per point (unfused form)
    bool curved = false;
    void *d_mu = nullptr, *d_mq = nullptr, *d_mfn = nullptr;
};

// Kernel ids for timing: 0..2 fused phases A, B, C; 10+k unfused kernel k (1..13); 30 RK4 update.
static cudaEvent_t pool_event(fr_mesh *m)
{
    if (!m->ev_pool.empty()) { cudaEvent_t e = m->ev_pool.back(); m->ev_pool.pop_back(); return e; }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

struct TimeScope {
    fr_mesh *m; int kernel; cudaStream_t s; cudaEvent_t a = nullptr;
    TimeScope(fr_mesh *m_, int k, cudaStream_t s_) : m(m_), kernel(k), s(s_)
    {
        if (m->timing) { a = pool_event(m); cudaEventRecord(a, s); }
    }
    ~TimeScope()
    {
        if (a) {
            cudaEvent_t b = pool_event(m);
            cudaEventRecord(b, s);
            m->timed.push_back({kernel, a, b});
        }
    }
};

static size_t tsize(int prec) { return prec == FR_FP64 ? sizeof(double) : sizeof(float); }

static fr_status dalloc(fr_mesh *m, void **p, size_t bytes)
{
    if (*p) return FR_OK;
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) { *p = nullptr; return fail(FR_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e)); }
    m->bytes += (long long)bytes;
    return FR_OK;
}

static void dfree(void *&p) { if (p) { cudaFree(p); p = nullptr; } }

// ---------------------------------------------------------------------------------------------
// Reference elements (hexahedra)
// ---------------------------------------------------------------------------------------------
static void hex_ref_fpts(const frb::Hex1D &h, std::vector<double> &xf)
{
    int n = h.n;
    xf.assign((size_t)6 * n * n * 3, 0.0);
    for (int f = 0; f < 6; f++) {
        int d = f / 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        for (int b = 0; b < n; b++)
            for (int a = 0; a < n; a++) {
                double *X = &xf[((size_t)f * n * n + a + n * b) * 3];
                X[d] = (f & 1) ? 1.0 : -1.0;
                X[t1] = h.x[a];
                X[t2] = h.x[b];
            }
    }
}

// Reference face quadrature points of a hexahedron: m x m GL points per face, same ordering as
// the flux points (local index a + m b over the face's two tangential directions).
static void hex_ref_qpts(int mq, std::vector<double> &xq)
{
    double x[FR_MAXM], w[FR_MAXM];
    frb::gauss_legendre(mq, x, w);
    xq.assign((size_t)6 * mq * mq * 3, 0.0);
    for (int f = 0; f < 6; f++) {
        int d = f / 2, t1 = d == 0 ? 1 : 0, t2 = d == 2 ? 1 : 2;
        for (int b = 0; b < mq; b++)
            for (int a = 0; a < mq; a++) {
                double *X = &xq[((size_t)f * mq * mq + a + mq * b) * 3];
                X[d] = (f & 1) ? 1.0 : -1.0;
                X[t1] = x[a];
                X[t2] = x[b];
            }
    }
}

// Reference flux points, face point counts and face centres of a block's element type.
struct RefFaces {
    int nfaces;
    int count[6], off[6];
    double centre[6][3];
    std::vector<double> xf;   // [nf][3]
};

static void ref_faces(const fr_mesh *m, int blk, RefFaces &r)
{
    const Block &B = m->blocks[blk];
    if (B.type == 0) {
        const frb::Hex1D &h = m->hex1d[blk];
        int n2 = h.n * h.n;
        r.nfaces = 6;
        hex_ref_fpts(h, r.xf);
        for (int f = 0; f < 6; f++) {
            r.count[f] = n2; r.off[f] = f * n2;
            r.centre[f][0] = r.centre[f][1] = r.centre[f][2] = 0.0;
            r.centre[f][f / 2] = (f & 1) ? 1.0 : -1.0;
        }
        return;
    }
    if (B.type == 2 || B.type == 3) {
        // dense types: faces from the operator tables; the centre of a face is the mean of its
        // vertices (a triangle's centroid, the base's centre)
        static const double tcen[4][3] = {{-1.0 / 3, -1.0 / 3, -1}, {-1.0 / 3, -1, -1.0 / 3}, {-1, -1.0 / 3, -1.0 / 3},
                                          {-1.0 / 3, -1.0 / 3, -1.0 / 3}};
        static const double ycen[5][3] = {{0, 0, -1}, {0, -2.0 / 3, -1.0 / 3}, {2.0 / 3, 0, -1.0 / 3}, {0, 2.0 / 3, -1.0 / 3},
                                          {-2.0 / 3, 0, -1.0 / 3}};
        const bool tet = B.type == 2;
        const int nfc = tet ? 4 : 5, nf = tet ? FR_TF : FR_YF;
        const int *foff = tet ? m->tet.foff : m->pyr.foff;
        r.nfaces = nfc;
        for (int f = 0; f < nfc; f++) {
            r.count[f] = foff[f + 1] - foff[f]; r.off[f] = foff[f];
            for (int d = 0; d < 3; d++) r.centre[f][d] = tet ? tcen[f][d] : ycen[f][d];
        }
        r.xf.assign((size_t)nf * 3, 0.0);
        for (int s2 = 0; s2 < nf; s2++)
            for (int d = 0; d < 3; d++) r.xf[(size_t)s2 * 3 + d] = tet ? m->tet.xf[s2][d] : m->pyr.xf[s2][d];
        return;
    }
    const frb::Prism2D &P = m->pri;
    static const int cnt[5] = {10, 10, 16, 16, 16};
    static const double cen[5][3] = {{-1.0 / 3, -1.0 / 3, -1}, {-1.0 / 3, -1.0 / 3, 1}, {0, -1, 0}, {0, 0, 0}, {-1, 0, 0}};
    r.nfaces = 5;
    int o = 0;
    for (int f = 0; f < 5; f++) {
        r.count[f] = cnt[f]; r.off[f] = o; o += cnt[f];
        for (int d = 0; d < 3; d++) r.centre[f][d] = cen[f][d];
    }
    r.xf.assign((size_t)68 * 3, 0.0);
    for (int t = 0; t < 10; t++)
        for (int f = 0; f < 2; f++) {
            double *X = &r.xf[(size_t)(f * 10 + t) * 3];
            X[0] = P.xt[t][0]; X[1] = P.xt[t][1]; X[2] = f ? 1.0 : -1.0;
        }
    for (int f = 0; f < 3; f++)
        for (int b = 0; b < 4; b++)
            for (int a = 0; a < 4; a++) {
                double *X = &r.xf[(size_t)(20 + 16 * f + a + 4 * b) * 3];
                double sp = P.z.x[a];
                if (f == 0) { X[0] = sp; X[1] = -1.0; }
                else if (f == 1) { X[0] = -sp; X[1] = sp; }
                else { X[0] = -1.0; X[1] = sp; }
                X[2] = P.z.x[b];
            }
}

static void affine_point(const double *x0J, const double *X, double *x)
{
    for (int i = 0; i < 3; i++) {
        x[i] = x0J[i];
        for (int j = 0; j < 3; j++) x[i] += x0J[3 + 3 * i + j] * (X[j] + 1.0);
    }
}

// Trilinear map of a hexahedron with vertices v[8][3] (tensor order, corner c at reference
// (+-1, +-1, +-1)): x(X) = sum_c N_c(X) v_c, N_c = prod_d (1 + s_cd X_d)/2, and J = dx/dX (row-major).
static void trilinear_map(const double *v, const double *X, double *x, double *J)
{
    if (x) x[0] = x[1] = x[2] = 0.0;
    if (J) for (int k = 0; k < 9; k++) J[k] = 0.0;
    for (int c = 0; c < 8; c++) {
        const double s0 = (c & 1) ? 1.0 : -1.0, s1 = (c & 2) ? 1.0 : -1.0, s2 = (c & 4) ? 1.0 : -1.0;
        const double f0 = 0.5 * (1.0 + s0 * X[0]), f1 = 0.5 * (1.0 + s1 * X[1]), f2 = 0.5 * (1.0 + s2 * X[2]);
        const double g[3] = {0.5 * s0 * f1 * f2, 0.5 * s1 * f0 * f2, 0.5 * s2 * f0 * f1};
        for (int i = 0; i < 3; i++) {
            if (x) x[i] += f0 * f1 * f2 * v[3 * c + i];
            if (J) for (int j = 0; j < 3; j++) J[3 * i + j] += g[j] * v[3 * c + i];
        }
    }
}

// Physical point of reference point X in element li of instance I (affine or trilinear map).
static void map_point(const struct InstanceHost &I, long long li, const double *X, double *x);

static double inv3(const double *a, double *b)
{
    double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    double id = 1.0 / det;
    b[0] = c00 * id; b[1] = (a[2] * a[7] - a[1] * a[8]) * id; b[2] = (a[1] * a[5] - a[2] * a[4]) * id;
    b[3] = c01 * id; b[4] = (a[0] * a[8] - a[2] * a[6]) * id; b[5] = (a[2] * a[3] - a[0] * a[5]) * id;
    b[6] = c02 * id; b[7] = (a[1] * a[6] - a[0] * a[7]) * id; b[8] = (a[0] * a[4] - a[1] * a[3]) * id;
    return det;
}

static void map_point(const InstanceHost &I, long long li, const double *X, double *x)
{
    if (!I.curved.empty() && I.curved[(size_t)li]) trilinear_map(&I.vx[(size_t)li * 24], X, x, nullptr);
    else affine_point(&I.x0J[(size_t)li * 12], X, x);
}

// ---------------------------------------------------------------------------------------------
// Face matching
// ---------------------------------------------------------------------------------------------
struct FaceRef {
    long long elem;   // global element
    int blk;          // block index
    long long le;     // element within block
    int face;
    double c[3];      // physical centroid
};

struct CellKey {
    long long i, j, k;
    bool operator==(const CellKey &o) const { return i == o.i && j == o.j && k == o.k; }
};
struct CellHash {
    size_t operator()(const CellKey &c) const
    {
        return (size_t)(c.i * 73856093LL) ^ (size_t)(c.j * 19349663LL) ^ (size_t)(c.k * 83492791LL);
    }
};

static double pdist2(const double *a, const double *b, const double *per)
{
    double s = 0;
    for (int d = 0; d < 3; d++) {
        double x = a[d] - b[d];
        if (per[d] > 0) x -= per[d] * std::nearbyint(x / per[d]);
        s += x * x;
    }
    return s;
}

// Builds partner codes for all flux points of one instance (its blocks are [b0, b1)).
static fr_status match_instance(fr_mesh *m, int ii, int b0, int b1, const fr_mesh_desc *d, std::vector<uint32_t> &partner)
{
    const InstanceHost &I = m->inst[ii];
    // element size scale for tolerances
    double hmin = 1e300;
    std::vector<FaceRef> faces;
    std::vector<RefFaces> rf(b1 - b0);
    for (int b = b0; b < b1; b++) {
        const Block &B = m->blocks[b];
        ref_faces(m, b, rf[b - b0]);
        for (long long le = 0; le < B.ne; le++) {
            const long long li = B.elem0 - m->blocks[b0].elem0 + le;
            const double *x0J = &I.x0J[(size_t)li * 12];
            double hh = std::cbrt(std::fabs(x0J[3] * (x0J[7] * x0J[11] - x0J[8] * x0J[10]) - x0J[4] * (x0J[6] * x0J[11] - x0J[8] * x0J[9]) + x0J[5] * (x0J[6] * x0J[10] - x0J[7] * x0J[9])));
            hmin = std::min(hmin, hh);
            for (int f = 0; f < rf[b - b0].nfaces; f++) {
                FaceRef fr;
                fr.elem = B.elem0 + le; fr.blk = b; fr.le = le; fr.face = f;
                map_point(I, li, rf[b - b0].centre[f], fr.c);
                faces.push_back(fr);
            }
        }
    }
    const double tol = 1e-7 * hmin, tol2 = tol * tol, cell = 8 * tol;
    long long ncell[3];
    for (int k = 0; k < 3; k++) ncell[k] = d->period[k] > 0 ? (long long)std::ceil(d->period[k] / cell) : 0;
    auto key_of = [&](const double *c) {
        long long q[3];
        for (int k = 0; k < 3; k++) {
            double x = c[k];
            if (d->period[k] > 0) x -= d->period[k] * std::floor(x / d->period[k]);
            q[k] = (long long)std::floor(x / cell);
            if (ncell[k] > 0) q[k] = ((q[k] % ncell[k]) + ncell[k]) % ncell[k];
        }
        return CellKey{q[0], q[1], q[2]};
    };
    std::unordered_map<CellKey, std::vector<int>, CellHash> open;
    std::vector<int> mate(faces.size(), -1);
    for (size_t a = 0; a < faces.size(); a++) {
        CellKey k0 = key_of(faces[a].c);
        int found = -1;
        for (int di = -1; di <= 1 && found < 0; di++)
            for (int dj = -1; dj <= 1 && found < 0; dj++)
                for (int dk = -1; dk <= 1 && found < 0; dk++) {
                    CellKey k{k0.i + di, k0.j + dj, k0.k + dk};
                    if (ncell[0]) k.i = ((k.i % ncell[0]) + ncell[0]) % ncell[0];
                    if (ncell[1]) k.j = ((k.j % ncell[1]) + ncell[1]) % ncell[1];
                    if (ncell[2]) k.k = ((k.k % ncell[2]) + ncell[2]) % ncell[2];
                    auto it = open.find(k);
                    if (it == open.end()) continue;
                    for (size_t t = 0; t < it->second.size(); t++) {
                        int b = it->second[t];
                        if (pdist2(faces[a].c, faces[b].c, d->period) < tol2) {
                            found = b;
                            it->second.erase(it->second.begin() + t);
                            break;
                        }
                    }
                }
        if (found >= 0) { mate[a] = found; mate[found] = (int)a; }
        else open[k0].push_back((int)a);
    }
    for (size_t a = 0; a < faces.size(); a++)
        if (mate[a] < 0)
            return fail(FR_EMESH, "instance %d: face %d of element %lld has no partner", ii, faces[a].face, faces[a].elem);
    // point permutations (cached per pair of face kinds)
    std::map<std::tuple<int, int, int, int>, std::vector<int>> perm_cache;
    std::vector<double> xa, xb;
    for (size_t a = 0; a < faces.size(); a++) {
        size_t b = (size_t)mate[a];
        if (b < a) continue;
        const FaceRef &A = faces[a], &Bf = faces[b];
        const Block &BA = m->blocks[A.blk], &BB = m->blocks[Bf.blk];
        const RefFaces &RA = rf[A.blk - b0], &RB = rf[Bf.blk - b0];
        int n2 = RA.count[A.face];
        if (RB.count[Bf.face] != n2) return fail(FR_EMESH, "element %lld face %d meets a face with a different point count", A.elem, A.face);
        const long long liA = A.elem - m->blocks[b0].elem0, liB = Bf.elem - m->blocks[b0].elem0;
        xa.resize(n2 * 3); xb.resize(n2 * 3);
        for (int t = 0; t < n2; t++) {
            map_point(I, liA, &RA.xf[((size_t)RA.off[A.face] + t) * 3], &xa[t * 3]);
            map_point(I, liB, &RB.xf[((size_t)RB.off[Bf.face] + t) * 3], &xb[t * 3]);
        }
        auto key = std::make_tuple(BA.type, A.face, BB.type, Bf.face);
        std::vector<int> &perm = perm_cache[key];
        bool ok = (int)perm.size() == n2;
        for (int t = 0; ok && t < n2; t++) ok = pdist2(&xa[t * 3], &xb[perm[t] * 3], d->period) < tol2;
        if (!ok) {
            perm.assign(n2, -1);
            for (int t = 0; t < n2; t++) {
                for (int u = 0; u < n2; u++)
                    if (pdist2(&xa[t * 3], &xb[u * 3], d->period) < tol2) { perm[t] = u; break; }
                if (perm[t] < 0) return fail(FR_EMESH, "flux point of element %lld face %d has no partner", A.elem, A.face);
            }
        }
        // reading R5: L is the smaller global element; a self-pair takes the smaller local face
        bool aL = A.elem < Bf.elem || (A.elem == Bf.elem && A.face < Bf.face);
        for (int t = 0; t < n2; t++) {
            long long ga = BA.f0 + A.le * BA.nf + RA.off[A.face] + t;
            long long gb = BB.f0 + Bf.le * BB.nf + RB.off[Bf.face] + perm[t];
            partner[ga] = (uint32_t)gb | (aL ? FR_LFLAG : 0u);
            partner[gb] = (uint32_t)ga | (aL ? 0u : FR_LFLAG);
        }
        m->npair += n2;
        if (m->surf) {
            // the same face pair on the m x m face quadrature points (single hexahedral block)
            const int mq = BA.m, q2 = mq * mq;
            static thread_local std::vector<double> refq;
            if ((int)refq.size() != 6 * q2 * 3) hex_ref_qpts(mq, refq);
            std::vector<double> qa(q2 * 3), qb(q2 * 3);
            for (int t = 0; t < q2; t++) {
                map_point(I, liA, &refq[((size_t)A.face * q2 + t) * 3], &qa[t * 3]);
                map_point(I, liB, &refq[((size_t)Bf.face * q2 + t) * 3], &qb[t * 3]);
            }
            auto qkey = std::make_tuple(-1, A.face, -1, Bf.face);
            std::vector<int> &qperm = perm_cache[qkey];
            bool qok = (int)qperm.size() == q2;
            for (int t = 0; qok && t < q2; t++) qok = pdist2(&qa[t * 3], &qb[qperm[t] * 3], d->period) < tol2;
            if (!qok) {
                qperm.assign(q2, -1);
                for (int t = 0; t < q2; t++) {
                    for (int u = 0; u < q2; u++)
                        if (pdist2(&qa[t * 3], &qb[u * 3], d->period) < tol2) { qperm[t] = u; break; }
                    if (qperm[t] < 0) return fail(FR_EMESH, "face quadrature point of element %lld face %d has no partner", A.elem, A.face);
                }
            }
            for (int t = 0; t < q2; t++) {
                long long ga = A.le * 6 * q2 + (long long)A.face * q2 + t;
                long long gb = Bf.le * 6 * q2 + (long long)Bf.face * q2 + qperm[t];
                m->qpartner_host[ga] = (uint32_t)gb | (aL ? FR_LFLAG : 0u);
                m->qpartner_host[gb] = (uint32_t)ga | (aL ? 0u : FR_LFLAG);
            }
        }
    }
    return FR_OK;
}

// ---------------------------------------------------------------------------------------------
// Mesh creation
// ---------------------------------------------------------------------------------------------
// Affine map of one element from its vertices; rejects non-affine and inverted elements.
// Affine map of one element from its vertices (x0J); a hexahedron that is not affine is kept as a
// trilinear (curved) element of instance I (local index li): its vertices are stored, and the
// element geometry recorded is the map's at the element centre. Other non-affine elements give
// FR_EUNSUPPORTED; inverted ones FR_EMESH.
static fr_status element_map(int ii, long long e, int type, const fr_mesh_desc *d, double *x0J, std::vector<double> &geo,
                             InstanceHost &I, long long li)
{
    const int nv = type == 0 ? 8 : (type == 1 ? 6 : (type == 2 ? 4 : 5));
    const int *conn = type == 0 ? d->hex_v + 8 * e
                      : type == 1 ? d->pri_v + 6 * e
                      : type == 2 ? d->tet_v + 4 * e
                                  : d->pyr_v + 5 * e;
    const double *v[8];
    for (int k = 0; k < nv; k++) {
        int vi = conn[k];
        if (vi < 0 || vi >= d->n_verts) return fail(FR_EMESH, "instance %d element %lld: vertex id %d out of range", ii, e, vi);
        v[k] = d->verts + 3 * (size_t)vi;
    }
    const int c3 = type == 0 ? 4 : 3;   // corner along the third reference axis (prisms, tetrahedra: v3)
    double scale = 0;
    for (int i = 0; i < 3; i++) {
        x0J[i] = v[0][i];
        x0J[3 + 3 * i + 0] = 0.5 * (v[1][i] - v[0][i]);
        x0J[3 + 3 * i + 1] = 0.5 * (v[2][i] - v[0][i]);
        // pyramid: the apex, reference (0,0,1), is corner 0 + (1,1,2) in reference units
        x0J[3 + 3 * i + 2] = type == 3 ? 0.5 * (v[4][i] - v[0][i]) - 0.25 * (v[1][i] - v[0][i]) - 0.25 * (v[2][i] - v[0][i])
                                       : 0.5 * (v[c3][i] - v[0][i]);
        scale = std::max(scale, std::fabs(v[1][i] - v[0][i]) + std::fabs(v[2][i] - v[0][i]) + std::fabs(v[type == 3 ? 4 : c3][i] - v[0][i]));
    }
    static const double pc[6][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {-1, 1, 1}};
    static const double pp[5][3] = {{-1, -1, -1}, {1, -1, -1}, {-1, 1, -1}, {1, 1, -1}, {0, 0, 1}};
    for (int k = 0; k < nv; k++) {  // affine: every corner is the image of its reference corner
        double X[3], x[3];
        if (type == 0) { X[0] = (k & 1) ? 1.0 : -1.0; X[1] = (k & 2) ? 1.0 : -1.0; X[2] = (k & 4) ? 1.0 : -1.0; }
        else if (type == 3) { X[0] = pp[k][0]; X[1] = pp[k][1]; X[2] = pp[k][2]; }
        else { X[0] = pc[k][0]; X[1] = pc[k][1]; X[2] = pc[k][2]; }
        affine_point(x0J, X, x);
        for (int i = 0; i < 3; i++)
            if (std::fabs(x[i] - v[k][i]) > 1e-10 * scale) {
                if (type != 0) return fail(FR_EUNSUPPORTED, "instance %d element %lld is not affine", ii, e);
                I.curved[(size_t)li] = 1;
            }
    }
    double Ji[9];
    double det;
    if (type == 0) {
        for (int k = 0; k < 8; k++)
            for (int i = 0; i < 3; i++) I.vx[(size_t)li * 24 + 3 * k + i] = v[k][i];
    }
    if (type == 0 && I.curved[(size_t)li]) {
        double J[9];
        const double X0[3] = {0.0, 0.0, 0.0};
        trilinear_map(&I.vx[(size_t)li * 24], X0, nullptr, J);
        det = inv3(J, Ji);
    } else {
        det = inv3(x0J + 3, Ji);
    }
    if (!(det > 0)) return fail(FR_EMESH, "instance %d element %lld is inverted or degenerate", ii, e);
    for (int k = 0; k < 9; k++) geo.push_back(Ji[k]);
    geo.push_back(det);
    return FR_OK;
}

static fr_status build_host(fr_mesh *m, const fr_mesh_desc *const *inst, int n_inst, const fr_params *prm,
                            std::vector<uint32_t> &partner)
{
    if (!inst || !prm || n_inst <= 0) return fail(FR_EINVAL, "null descriptor or n_inst <= 0");
    m->prec = prm[0].prec;
    if (m->prec < FR_FP64 || m->prec > FR_MIXED_FP16) return fail(FR_EINVAL, "unknown precision %d", m->prec);
    long long elem = 0, u = 0, f = 0;
    std::vector<int> bfirst;
    for (int ii = 0; ii < n_inst; ii++) {
        const fr_mesh_desc *d = inst[ii];
        const fr_params &P = prm[ii];
        if (!d) return fail(FR_EINVAL, "instance %d: null descriptor", ii);
        if (P.prec != m->prec) return fail(FR_EINVAL, "all instances must share one precision");
        int m1 = P.nq1d > 0 ? P.nq1d : P.p + 2;
        // m1 = p + 2: flux anti-aliasing on (p + 2)^3 GL points; m1 = p + 1: the quadrature points are
        // the solution points, i.e. the collocation form without anti-aliasing (hexahedra only)
        if (P.p < 3 || P.p > 4 || (m1 != P.p + 2 && m1 != P.p + 1))
            return fail(FR_EUNSUPPORTED, "instance %d: order %d with %d quadrature points", ii, P.p, m1);
        if (m1 == P.p + 1 && d && (d->n_pri > 0 || d->n_tet > 0 || d->n_pyr > 0))
            return fail(FR_EUNSUPPORTED, "instance %d: prisms, tetrahedra and pyramids are built with flux anti-aliasing only", ii);
        if (P.surface_aa) {
            if (n_inst != 1 || !d || d->n_pri > 0 || d->n_tet > 0 || d->n_pyr > 0 || m1 != P.p + 2)
                return fail(FR_EUNSUPPORTED, "surface-flux anti-aliasing runs single-instance hexahedral meshes with m = p + 2");
            m->surf = true;
        }
        if (!(P.gamma > 1.0) || !(P.Pr > 0.0) || P.mu < 0.0 || P.tau < 0.0 || !(P.p_ref == P.p_ref) ||
            !(P.rho_ref >= 0.0))
            return fail(FR_EINVAL, "instance %d: bad physical parameters", ii);
        if (P.rusanov_mode != 0) return fail(FR_EUNSUPPORTED, "rusanov_mode %d", P.rusanov_mode);
        if (d->n_hex < 0 || d->n_pri < 0 || d->n_tet < 0 || d->n_pyr < 0 || d->n_hex + d->n_pri + d->n_tet + d->n_pyr == 0 ||
            d->n_verts <= 0 || !d->verts)
            return fail(FR_EINVAL, "instance %d: empty or malformed mesh", ii);
        if (d->n_hex > 0 && !d->hex_v) return fail(FR_EINVAL, "instance %d: null hex connectivity", ii);
        if (d->n_pri > 0 && !d->pri_v) return fail(FR_EINVAL, "instance %d: null prism connectivity", ii);
        if (d->n_tet > 0 && !d->tet_v) return fail(FR_EINVAL, "instance %d: null tetrahedron connectivity", ii);
        if (d->n_tet > 0 && P.p != 3)
            return fail(FR_EUNSUPPORTED, "instance %d: tetrahedra are built for p = 3", ii);
        if (d->n_pyr > 0 && !d->pyr_v) return fail(FR_EINVAL, "instance %d: null pyramid connectivity", ii);
        if (d->n_pyr > 0 && P.p != 3)
            return fail(FR_EUNSUPPORTED, "instance %d: pyramids are built for p = 3", ii);

        if (d->n_pri > 0 && (P.p != 3 || (P.tri_strength != 0 && P.tri_strength != 8)))
            return fail(FR_EUNSUPPORTED, "instance %d: prisms are built for p = 3 with a strength-8 triangle rule", ii);
        InstanceHost I;
        I.prm = P; I.prm.nq1d = m1;
        I.n_hex = d->n_hex; I.n_pri = d->n_pri; I.n_tet = d->n_tet; I.n_pyr = d->n_pyr;
        const size_t nel = (size_t)d->n_hex + d->n_pri + d->n_tet + d->n_pyr;
        I.x0J.resize(nel * 12);
        I.curved.assign(nel, 0);
        I.vx.assign(nel * 24, 0.0);
        m->inst_u0.push_back(u);
        bfirst.push_back((int)m->blocks.size());
        for (int type = 0; type < 4; type++) {
            long long ne = type == 0 ? d->n_hex : (type == 1 ? d->n_pri : (type == 2 ? d->n_tet : d->n_pyr));
            if (ne == 0) continue;
            Block B{};
            B.inst = ii; B.type = type; B.p = P.p; B.m = m1;
            frb::Hex1D h;
            if (type == 0) {
                // the device tables hold the p + 2 point operators (the collocation form uses none of
                // the quadrature-point ones)
                if (frb::hex1d(P.p, P.p + 2, h)) return fail(FR_EUNSUPPORTED, "hex operators for p=%d", P.p);
                B.nu = (P.p + 1) * (P.p + 1) * (P.p + 1); B.nf = 6 * (P.p + 1) * (P.p + 1);
            } else if (type == 1) {
                if (!m->has_pri) {
                    if (frb::prism2d(m->pri)) return fail(FR_EUNSUPPORTED, "prism operators");
                    m->has_pri = true;
                }
                h = m->pri.z;
                B.nu = FR_PT * FR_PE; B.nf = 2 * FR_PT + 3 * FR_PE * FR_PE;
            } else if (type == 2) {
                if (!m->has_tet) {
                    if (frb::tet3d(m->tet)) return fail(FR_EUNSUPPORTED, "tetrahedron operators");
                    m->has_tet = true;
                }
                std::memset(&h, 0, sizeof h);
                B.nu = FR_TU; B.nf = FR_TF;
            } else {
                if (!m->has_pyr) {
                    if (frb::pyr3d(m->pyr)) return fail(FR_EUNSUPPORTED, "pyramid operators");
                    m->has_pyr = true;
                }
                std::memset(&h, 0, sizeof h);
                B.nu = FR_YU; B.nf = FR_YF;
            }
            B.ne = ne; B.elem0 = elem; B.u0 = u; B.f0 = f;
            long long le0 = type == 0 ? 0 : (type == 1 ? d->n_hex : (type == 2 ? d->n_hex + d->n_pri : d->n_hex + d->n_pri + d->n_tet));
            for (long long e = 0; e < ne; e++) {
                fr_status st = element_map(ii, e, type, d, &I.x0J[(size_t)(le0 + e) * 12], m->geo_host, I, le0 + e);
                if (st) return st;
            }
            m->blocks.push_back(B);
            m->hex1d.push_back(h);
            elem += B.ne; u += B.ne * FR_NV * B.nu; f += B.ne * B.nf;
        }
        m->inst.push_back(I);
    }
    m->ne = elem; m->nU = u; m->nfpt = f;
    for (const InstanceHost &I : m->inst)
        for (char c : I.curved) m->curved = m->curved || c;
    if (m->curved && (n_inst != 1 || m->blocks.size() != 1 || m->surf || m->blocks[0].m != m->blocks[0].p + 2))
        return fail(FR_EUNSUPPORTED, "curved (non-affine) hexahedra run single-instance hexahedral meshes with flux "
                                     "anti-aliasing (m = p + 2)");
    m->inst_u0.push_back(u);
    bfirst.push_back((int)m->blocks.size());
    if (f >= (long long)FR_LFLAG) return fail(FR_EUNSUPPORTED, "more than 2^31 flux points");
    partner.assign((size_t)f, 0xffffffffu);
    if (m->surf) {
        const Block &B = m->blocks[0];
        m->nqf = B.ne * 6LL * B.m * B.m;
        if (m->nqf >= (long long)FR_LFLAG) return fail(FR_EUNSUPPORTED, "more than 2^31 face quadrature points");
        m->qpartner_host.assign((size_t)m->nqf, 0xffffffffu);
    }
    for (int ii = 0; ii < n_inst; ii++) {
        fr_status st = match_instance(m, ii, bfirst[ii], bfirst[ii + 1], inst[ii], partner);
        if (st != FR_OK) return st;
    }
    return FR_OK;
}

template <typename T>
static void fill_priops(const frb::Prism2D &P, PriOps<T> &o)
{
    o = PriOps<T>{};
    for (int q = 0; q < FR_PQ; q++)
        for (int t = 0; t < FR_PT; t++) { o.Bt[q][t] = (T)P.Bt[q][t]; o.Pt[t][q] = (T)P.Pt[t][q]; }
    for (int t = 0; t < FR_PT; t++)
        for (int u = 0; u < FR_PT; u++) { o.Dhx[t][u] = (T)P.Dhx[t][u]; o.Dhy[t][u] = (T)P.Dhy[t][u]; }
    for (int f = 0; f < 3; f++) {
        o.nf[f][0] = (T)P.nf[f][0]; o.nf[f][1] = (T)P.nf[f][1];
        for (int a = 0; a < FR_PE; a++)
            for (int t = 0; t < FR_PT; t++) { o.Ef[f][a][t] = (T)P.Ef[f][a][t]; o.Lf[f][t][a] = (T)P.Lf[f][t][a]; }
    }
    for (int c = 0; c < 5; c++)
        for (int k = 0; k < FR_PE; k++) { o.Bz[c][k] = (T)P.z.B[c][k]; o.Pz[k][c] = (T)P.z.Pj[k][c]; }
    for (int k = 0; k < FR_PE; k++) {
        for (int j = 0; j < FR_PE; j++) o.Dhz[k][j] = (T)P.z.Dh[k][j];
        o.lzL[k] = (T)P.z.lL[k]; o.lzR[k] = (T)P.z.lR[k]; o.liftzL[k] = (T)P.z.liftL[k]; o.liftzR[k] = (T)P.z.liftR[k];
    }
}

template <typename T>
static fr_status upload_priops(fr_mesh *m, void **dst)
{
    if (!m->has_pri) return FR_OK;
    PriOps<T> o;
    fill_priops<T>(m->pri, o);
    fr_status st = dalloc(m, dst, sizeof(o));
    if (st) return st;
    CU(cudaMemcpy(*dst, &o, sizeof(o), cudaMemcpyHostToDevice));
    if constexpr (sizeof(T) == 4) {
        // the FP32 volume kernels read the interpolation and projection blocks from constant memory
        if (pri_set_const_ops(&o) || multi_set_pri_const_ops(&o)) return fail(FR_ECUDA, "prism operator upload failed");
    }
    return FR_OK;
}

// Transposed dense-element operator tables (DenseOps) from the host construction (DenseRef).
template <typename T, typename REF, typename OPS>
static fr_status upload_dense(fr_mesh *m, const REF &R, void **dst)
{
    constexpr int NU = REF::NU, NF = REF::NF, NFACE = REF::NFACE;
    std::vector<OPS> o(1);   // value-initialised: the pad rows stay zero
    OPS &t = o[0];
    for (int j = 0; j < NU; j++) {
        for (int q = 0; q < FR_TQ; q++) t.Bt[j][q] = (T)R.B[q][j];
        for (int s2 = 0; s2 < NF; s2++) t.M0t[j][s2] = (T)R.M0[s2][j];
        for (int d = 0; d < 3; d++)
            for (int z = 0; z < NU; z++) t.Dht[d][j][z] = (T)R.Dh[d][z][j];
    }
    for (int s2 = 0; s2 < NF; s2++)
        for (int z = 0; z < NU; z++) t.Lt[s2][z] = (T)R.L[z][s2];
    // projection with the corrected divergence: (Dh_d Pj)[z][q], formed in FP64
    for (int d = 0; d < 3; d++)
        for (int q = 0; q < FR_TQ; q++)   // rows FR_TQ .. FR_TQP-1 stay zero
            for (int z = 0; z < NU; z++) {
                double v = 0;
                for (int j = 0; j < NU; j++) v += R.Dh[d][z][j] * R.Pj[j][q];
                t.Dvt[d][q][z] = (T)v;
            }
    for (int f = 0; f < NFACE; f++)
        for (int d = 0; d < 3; d++) t.nf[f][d] = (T)R.nf[f][d];
    for (int f = 0; f <= NFACE; f++) {
        t.foff[f] = R.foff[f];
        if (R.foff[f] != (f == NFACE ? NF : OPS::F0(f))) return fail(FR_EUNSUPPORTED, "dense-element face layout");
    }
    fr_status st = dalloc(m, dst, sizeof(OPS));
    if (st) return st;
    CU(cudaMemcpy(*dst, o.data(), sizeof(OPS), cudaMemcpyHostToDevice));
    return FR_OK;
}

// Float-float copy of the dense tables the low-Mach form's mass channel reads (M0, Dh, L):
// hi = float(op), lo = float(op - hi).
// The low-Mach geometry of one element from its FP64 inverse Jacobian and determinant (10 values).
static GeoLM geo_lm(const double *src)
{
    GeoLM x;
    for (int k = 0; k < 9; k++) x.Ji[k] = src[k];
    x.det = src[9];
    for (int k = 0; k < 9; k++) x.cm[k] = ff_from_double(x.det * x.Ji[k]);
    x.idet = ff_from_double(-1.0 / x.det);
    return x;
}

template <typename REF, typename OPSF>
static fr_status upload_dense_ff(fr_mesh *m, const REF &R, void **dst)
{
    constexpr int NU = REF::NU, NF = REF::NF;
    std::vector<DenseOpsFF<OPSF>> o(1);   // value-initialised
    OPSF &h = o[0].hi, &l = o[0].lo;
    auto split = [](double v, float &hi, float &lo) { hi = (float)v; lo = (float)(v - (double)hi); };
    for (int j = 0; j < NU; j++) {
        for (int s2 = 0; s2 < NF; s2++) split(R.M0[s2][j], h.M0t[j][s2], l.M0t[j][s2]);
        for (int d = 0; d < 3; d++)
            for (int z = 0; z < NU; z++) {
                split(R.Dh[d][z][j], h.Dht[d][j][z], l.Dht[d][j][z]);
                o[0].Dht64[d][j][z] = R.Dh[d][z][j];
            }
    }
    for (int s2 = 0; s2 < NF; s2++)
        for (int z = 0; z < NU; z++) split(R.L[z][s2], h.Lt[s2][z], l.Lt[s2][z]);
    fr_status st = dalloc(m, dst, sizeof(DenseOpsFF<OPSF>));
    if (st) return st;
    CU(cudaMemcpy(*dst, o.data(), sizeof(DenseOpsFF<OPSF>), cudaMemcpyHostToDevice));
    return FR_OK;
}

template <typename T>
static fr_status upload_dense_tables(fr_mesh *m)
{
    fr_status st = FR_OK;
    if (m->has_tet) st = upload_dense<T, frb::Tet3D, TetOps<T>>(m, m->tet, &m->d_tetops);
    if (!st && m->has_pyr) st = upload_dense<T, frb::Pyr3D, PyrOps<T>>(m, m->pyr, &m->d_pyrops);
    return st;
}

template <typename T>
static fr_status upload_curved(fr_mesh *m)
{
    if (!m->curved) return FR_OK;
    const Block &B = m->blocks[0];
    const InstanceHost &I = m->inst[0];
    const frb::Hex1D &h = m->hex1d[0];
    const int n = h.n, mq = h.m, nu = B.nu, nf = B.nf, nq = mq * mq * mq;
    std::vector<double> xf;
    hex_ref_fpts(h, xf);
    std::vector<T> tu((size_t)B.ne * nu * 10), tq((size_t)B.ne * nq * 9), tf((size_t)B.ne * nf * 4);
    for (long long e = 0; e < B.ne; e++) {
        const double *v = &I.vx[(size_t)e * 24];
        double J[9], Ji[9], det;
        for (int z = 0; z < nu; z++) {
            const double X[3] = {h.x[z % n], h.x[(z / n) % n], h.x[z / (n * n)]};
            trilinear_map(v, X, nullptr, J);
            det = inv3(J, Ji);
            if (!(det > 0)) return fail(FR_EMESH, "curved element %lld is not invertible at a solution point", e);
            for (int k = 0; k < 9; k++) tu[((size_t)e * nu + z) * 10 + k] = (T)Ji[k];
            tu[((size_t)e * nu + z) * 10 + 9] = (T)det;
        }
        for (int q = 0; q < nq; q++) {
            const double X[3] = {h.xq[q % mq], h.xq[(q / mq) % mq], h.xq[q / (mq * mq)]};
            trilinear_map(v, X, nullptr, J);
            det = inv3(J, Ji);
            if (!(det > 0)) return fail(FR_EMESH, "curved element %lld is not invertible at a quadrature point", e);
            for (int k = 0; k < 9; k++) tq[((size_t)e * nq + q) * 9 + k] = (T)(det * Ji[k]);
        }
        for (int s2 = 0; s2 < nf; s2++) {
            const int f = s2 / (n * n);
            trilinear_map(v, &xf[(size_t)s2 * 3], nullptr, J);
            det = inv3(J, Ji);
            if (!(det > 0)) return fail(FR_EMESH, "curved element %lld is not invertible at a flux point", e);
            double nr[3] = {0, 0, 0}, ns[3];
            nr[f / 2] = (f & 1) ? 1.0 : -1.0;
            for (int k = 0; k < 3; k++) ns[k] = det * (Ji[k] * nr[0] + Ji[3 + k] * nr[1] + Ji[6 + k] * nr[2]);
            const double mag = std::sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
            for (int k = 0; k < 3; k++) tf[((size_t)e * nf + s2) * 4 + k] = (T)(ns[k] / mag);
            tf[((size_t)e * nf + s2) * 4 + 3] = (T)mag;
        }
    }
    fr_status st = dalloc(m, &m->d_mu, tu.size() * sizeof(T));
    if (!st) st = dalloc(m, &m->d_mq, tq.size() * sizeof(T));
    if (!st) st = dalloc(m, &m->d_mfn, tf.size() * sizeof(T));
    if (st) return st;
    CU(cudaMemcpy(m->d_mu, tu.data(), tu.size() * sizeof(T), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(m->d_mq, tq.data(), tq.size() * sizeof(T), cudaMemcpyHostToDevice));
    CU(cudaMemcpy(m->d_mfn, tf.data(), tf.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FR_OK;
}

template <typename T>
static fr_status upload_geo(fr_mesh *m)
{
    std::vector<Geo<T>> g((size_t)m->ne);
    for (long long e = 0; e < m->ne; e++) {
        for (int k = 0; k < 9; k++) g[e].Ji[k] = (T)m->geo_host[(size_t)e * 10 + k];
        g[e].det = (T)m->geo_host[(size_t)e * 10 + 9];
        g[e].nidet = T(-1) / g[e].det;
    }
    fr_status st = dalloc(m, &m->d_geo, g.size() * sizeof(Geo<T>));
    if (st) return st;
    CU(cudaMemcpy(m->d_geo, g.data(), g.size() * sizeof(Geo<T>), cudaMemcpyHostToDevice));
    return FR_OK;
}

template <typename T>
static Phys<T> phys_of(const fr_params &P)
{
    Phys<T> ph;
    ph.gamma = (T)P.gamma; ph.gm1 = (T)(P.gamma - 1.0); ph.mu = (T)P.mu;
    ph.beta = (T)P.beta; ph.tau = (T)P.tau; ph.heat = (T)(P.mu * P.gamma / P.Pr); ph.pref = (T)P.p_ref;
    ph.dev = 0;
    ph.rref = (T)P.rho_ref; ph.eref = (T)(P.p_ref / (P.gamma - 1.0));
    ph.rrefd = P.rho_ref;
    ph.H0d = P.rho_ref > 0 ? P.gamma * P.p_ref / ((P.gamma - 1.0) * P.rho_ref) : 0.0;
    ph.H0 = (T)ph.H0d;
    ph.H0ff = ff_from_double(ph.H0d);
    return ph;
}

// Unit outward normal and |n_s| (n_s = detJ J^-T n~) of every face of every element, in FP64.
static void build_face_normals(fr_mesh *m)
{
    const double r2 = 1.0 / std::sqrt(2.0);
    const double pri_n[5][3] = {{0, 0, -1}, {0, 0, 1}, {0, -1, 0}, {r2, r2, 0}, {-1, 0, 0}};
    m->fnrm_host.assign((size_t)m->ne * 24, 0.0);
    for (const Block &B : m->blocks)
        for (long long e = 0; e < B.ne; e++) {
            const long long ge = B.elem0 + e;
            const double *Ji = &m->geo_host[(size_t)ge * 10], det = m->geo_host[(size_t)ge * 10 + 9];
            const int nfaces = B.type == 0 ? 6 : (B.type == 1 ? 5 : (B.type == 2 ? 4 : 5));
            for (int f = 0; f < nfaces; f++) {
                double nr[3] = {0, 0, 0};
                if (B.type == 0) nr[f / 2] = (f & 1) ? 1.0 : -1.0;
                else if (B.type == 1) for (int d = 0; d < 3; d++) nr[d] = pri_n[f][d];
                else if (B.type == 2) for (int d = 0; d < 3; d++) nr[d] = m->tet.nf[f][d];
                else for (int d = 0; d < 3; d++) nr[d] = m->pyr.nf[f][d];
                double ns[3];
                for (int k = 0; k < 3; k++) ns[k] = det * (Ji[k] * nr[0] + Ji[3 + k] * nr[1] + Ji[6 + k] * nr[2]);
                const double mag = std::sqrt(ns[0] * ns[0] + ns[1] * ns[1] + ns[2] * ns[2]);
                double *o = &m->fnrm_host[((size_t)ge * 6 + f) * 4];
                for (int k = 0; k < 3; k++) o[k] = ns[k] / mag;
                o[3] = mag;
            }
        }
}

template <typename T>
static fr_status upload_face_normals(fr_mesh *m, const std::vector<long long> &order, void **dT, double **d64)
{
    std::vector<T> t(order.size() * 24);
    std::vector<ff> t64(order.size() * 24);   // float-float copy for the low-Mach mass channel
    for (size_t i = 0; i < order.size(); i++)
        for (int k = 0; k < 24; k++) {
            const double v = m->fnrm_host[(size_t)order[i] * 24 + k];
            t64[i * 24 + k] = ff_from_double(v);
            t[i * 24 + k] = (T)v;
        }
    fr_status st = dalloc(m, dT, t.size() * sizeof(T));
    if (st) return st;
    CU(cudaMemcpy(*dT, t.data(), t.size() * sizeof(T), cudaMemcpyHostToDevice));
    if (m->lowmach) {
        st = dalloc(m, (void **)d64, t64.size() * sizeof(ff));
        if (st) return st;
        CU(cudaMemcpy(*d64, t64.data(), t64.size() * sizeof(ff), cudaMemcpyHostToDevice));
    }
    return FR_OK;
}

template <typename T>
static fr_status build_groups(fr_mesh *m, const std::vector<uint32_t> &partner)
{
    {
        build_face_normals(m);
        std::vector<long long> all((size_t)m->ne);
        for (long long e = 0; e < m->ne; e++) all[e] = e;
        fr_status st = upload_face_normals<T>(m, all, &m->d_fnrm, &m->d_fnrm64);
        if (st) return st;
    }
    for (size_t b = 0; b < m->blocks.size(); b++) {
        const Block &B = m->blocks[b];
        Group *g = nullptr;
        for (Group &x : m->groups) if (x.type == B.type && x.p == B.p && x.m == B.m) g = &x;
        if (!g) { m->groups.push_back(Group()); g = &m->groups.back(); g->type = B.type; g->p = B.p; g->m = B.m; }
        g->blks.push_back((int)b);
        g->ne += B.ne;
    }
    std::vector<Phys<T>> tab;
    for (const InstanceHost &I : m->inst) {
        tab.push_back(phys_of<T>(I.prm));
        tab.back().dev = m->lowmach ? 1 : 0;
    }
    for (Group &g : m->groups) {
        // L points for the split interface phase
        std::vector<uint32_t> lp;
        long long eg = 0;
        for (int bi : g.blks) {
            const Block &B = m->blocks[bi];
            for (long long e = 0; e < B.ne; e++, eg++)
                for (int sp = 0; sp < B.nf; sp++)
                    if (partner[(size_t)(B.f0 + e * B.nf + sp)] & FR_LFLAG) lp.push_back((uint32_t)(eg * 256 + sp));
        }
        if (eg >= (1LL << 24)) return fail(FR_EUNSUPPORTED, "more than 2^24 elements of one type and order");
        g.nlpts = (long long)lp.size();
        fr_status sl = dalloc(m, (void **)&g.d_lpts, lp.size() * sizeof(uint32_t));
        if (sl) return sl;
        CU(cudaMemcpy(g.d_lpts, lp.data(), lp.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
        if (g.blks.size() < 2) continue;
        {
            std::vector<long long> order;
            for (int bi : g.blks)
                for (long long e = 0; e < m->blocks[bi].ne; e++) order.push_back(m->blocks[bi].elem0 + e);
            fr_status sn = upload_face_normals<T>(m, order, &g.d_fnrm, &g.d_fnrm64);
            if (sn) return sn;
        }
        if (m->lowmach) {
            std::vector<GeoLM> g64;
            for (int bi : g.blks) {
                const Block &B = m->blocks[bi];
                for (long long e = 0; e < B.ne; e++) g64.push_back(geo_lm(&m->geo_host[(size_t)(B.elem0 + e) * 10]));
            }
            fr_status sg = dalloc(m, &g.d_geo64, g64.size() * sizeof(GeoLM));
            if (sg) return sg;
            CU(cudaMemcpy(g.d_geo64, g64.data(), g64.size() * sizeof(GeoLM), cudaMemcpyHostToDevice));
        }
        std::vector<Geo<T>> geo;
        std::vector<long long> eu0, ef0;
        std::vector<int> eph;
        for (int bi : g.blks) {
            const Block &B = m->blocks[bi];
            for (long long e = 0; e < B.ne; e++) {
                Geo<T> x;
                const double *src = &m->geo_host[(size_t)(B.elem0 + e) * 10];
                for (int k = 0; k < 9; k++) x.Ji[k] = (T)src[k];
                x.det = (T)src[9];
                x.nidet = T(-1) / x.det;
                geo.push_back(x);
                eu0.push_back(B.u0 + e * FR_NV * B.nu);
                ef0.push_back(B.f0 + e * B.nf);
                eph.push_back(B.inst);
            }
        }
        fr_status st = dalloc(m, &g.d_geo, geo.size() * sizeof(Geo<T>));
        if (!st) st = dalloc(m, (void **)&g.d_eu0, eu0.size() * sizeof(long long));
        if (!st) st = dalloc(m, (void **)&g.d_ef0, ef0.size() * sizeof(long long));
        if (!st) st = dalloc(m, (void **)&g.d_eph, eph.size() * sizeof(int));
        if (!st) st = dalloc(m, &g.d_phtab, tab.size() * sizeof(Phys<T>));
        if (st) return st;
        CU(cudaMemcpy(g.d_geo, geo.data(), geo.size() * sizeof(Geo<T>), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(g.d_eu0, eu0.data(), eu0.size() * sizeof(long long), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(g.d_ef0, ef0.data(), ef0.size() * sizeof(long long), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(g.d_eph, eph.data(), eph.size() * sizeof(int), cudaMemcpyHostToDevice));
        CU(cudaMemcpy(g.d_phtab, tab.data(), tab.size() * sizeof(Phys<T>), cudaMemcpyHostToDevice));
    }
    return FR_OK;
}

static cudaError_t diag_scratch_lookup(int dev);

// Uploads everything a handle built on the host needs on the current device (m is deleted on failure).
static fr_status finish_create(fr_mesh *m, std::vector<uint32_t> &partner, fr_mesh **out);

extern "C" fr_status fr_mesh_create(const fr_mesh_desc *const *inst, int n_inst, const fr_params *prm, fr_mesh **out)
{
    if (!out) return fail(FR_EINVAL, "out is null");
    *out = nullptr;
    fr_mesh *m = new fr_mesh();
    std::vector<uint32_t> partner;
    fr_status st = build_host(m, inst, n_inst, prm, partner);
    if (st) { delete m; return st; }
    m->nfpt_own = m->nfpt;
    m->E1 = m->ne;
    return finish_create(m, partner, out);
}

static fr_status finish_create(fr_mesh *m, std::vector<uint32_t> &partner, fr_mesh **out)
{
    fr_status st = FR_OK;
    cudaError_t ce = cudaGetDevice(&m->dev);
    if (ce != cudaSuccess) { delete m; return fail(FR_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(ce)); }
    ce = cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, m->dev);
    if (ce != cudaSuccess || m->nsm < 1) { delete m; return fail(FR_ECUDA, "cudaDeviceGetAttribute: %s", cudaGetErrorString(ce)); }
    // the device address of the fixed diagnostics array (fr_diagnostics_noalloc), looked up afresh for
    // every handle so that it stays valid across a cudaDeviceReset
    if (diag_scratch_lookup(m->dev) != cudaSuccess) { delete m; return fail(FR_ECUDA, "cudaGetSymbolAddress failed"); }
    for (size_t b = 0; b < m->blocks.size(); b++)
        if (m->blocks[b].type == 0 && hex_upload_ops(m->blocks[b].p, m->blocks[b].p + 2, m->hex1d[b])) { delete m; return fail(FR_ECUDA, "operator upload failed"); }
    size_t ts = tsize(m->prec);
    st = (m->prec == FR_FP64) ? upload_geo<double>(m) : upload_geo<float>(m);
    if (!st) st = (m->prec == FR_FP64) ? upload_priops<double>(m, &m->d_priops) : upload_priops<float>(m, &m->d_priops);
    if (!st) st = (m->prec == FR_FP64) ? upload_dense_tables<double>(m) : upload_dense_tables<float>(m);
    if (!st) st = (m->prec == FR_FP64) ? upload_curved<double>(m) : upload_curved<float>(m);
    if (!st && m->prec != FR_FP64) {
        bool all = true;
        for (const InstanceHost &I : m->inst) all = all && I.prm.p_ref > 0 && I.prm.rho_ref > 0;
        m->lowmach = all;
    }
    if (!st && m->prec != FR_FP64 && m->has_pri) {
        // float-float prism operators for the mass channel: hi = float(op), lo = float(op - hi)
        PriOps<double> o64;
        fill_priops<double>(m->pri, o64);
        PriOpsFF pff{};
        fill_priops<float>(m->pri, pff.hi);
        const double *src = reinterpret_cast<const double *>(&o64);
        const float *h = reinterpret_cast<const float *>(&pff.hi);
        float *l = reinterpret_cast<float *>(&pff.lo);
        static_assert(sizeof(PriOps<double>) == 2 * sizeof(PriOps<float>), "same member layout in both precisions");
        for (size_t i = 0; i < sizeof(PriOps<float>) / sizeof(float); i++) l[i] = (float)(src[i] - (double)h[i]);
        st = dalloc(m, &m->d_priops64, sizeof(pff));
        if (!st && cudaMemcpy(m->d_priops64, &pff, sizeof(pff), cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(FR_ECUDA, "prism operator upload failed");
    }
    // float-float dense tables: the compensated face values of every reduced precision, and the
    // low-Mach form's mass channel
    if (!st && m->prec != FR_FP64 && m->has_tet) st = upload_dense_ff<frb::Tet3D, TetOps<float>>(m, m->tet, &m->d_tetops64);
    if (!st && m->prec != FR_FP64 && m->has_pyr) st = upload_dense_ff<frb::Pyr3D, PyrOps<float>>(m, m->pyr, &m->d_pyrops64);
    if (!st && m->lowmach) {
        std::vector<GeoLM> g64((size_t)m->ne);
        for (long long e = 0; e < m->ne; e++) g64[e] = geo_lm(&m->geo_host[(size_t)e * 10]);
        st = dalloc(m, &m->d_geo64, g64.size() * sizeof(GeoLM));
        if (!st && cudaMemcpy(m->d_geo64, g64.data(), g64.size() * sizeof(GeoLM), cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(FR_ECUDA, "geometry upload failed");
        if (!st) st = dalloc(m, (void **)&m->d_MF, (size_t)m->nfpt * sizeof(ff));
        if (!st) st = dalloc(m, (void **)&m->d_RL, (size_t)(m->nU / FR_NV) * sizeof(ff));
    }
    if (!st) st = (m->prec == FR_FP64) ? build_groups<double>(m, partner) : build_groups<float>(m, partner);
    // FP64 hexahedral handles evaluate each interface pair once (split interface phase)
    // (a partitioned handle evaluates each side's own points: the pair's other side may be remote)
    m->split_c = (((m->prec == FR_FP64) && !m->has_pri && !m->has_tet && !m->has_pyr) || m->surf) && m->nparts == 1;
    if (!st && m->surf) {
        std::vector<uint32_t> ql;
        for (long long q = 0; q < m->nqf; q++)
            if (m->qpartner_host[(size_t)q] & FR_LFLAG) ql.push_back((uint32_t)q);
        m->nqlpts = (long long)ql.size();
        st = dalloc(m, (void **)&m->d_qlpts, ql.size() * sizeof(uint32_t));
        if (!st && cudaMemcpy(m->d_qlpts, ql.data(), ql.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(FR_ECUDA, "face quadrature list upload failed");
        if (!st) st = dalloc(m, &m->d_DQ, (size_t)5 * m->nqf * ts);
    }
    if (!st && m->surf) {
        st = dalloc(m, (void **)&m->d_qpartner, m->qpartner_host.size() * sizeof(uint32_t));
        if (!st && cudaMemcpy(m->d_qpartner, m->qpartner_host.data(), m->qpartner_host.size() * sizeof(uint32_t),
                              cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(FR_ECUDA, "face quadrature partner upload failed");
        if (!st) st = dalloc(m, &m->d_UFQ, (size_t)5 * m->nqf * ts);
        if (!st) st = dalloc(m, &m->d_FVQ, (size_t)4 * m->nqf * ts);
    }
    if (!st && m->split_c) st = dalloc(m, &m->d_DF, (size_t)5 * m->nfpt * ts);
    if (!st) st = dalloc(m, (void **)&m->d_partner, partner.size() * sizeof(uint32_t));
    if (!st && cudaMemcpy(m->d_partner, partner.data(), partner.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess)
        st = fail(FR_ECUDA, "partner upload failed");
    if (!st) st = dalloc(m, &m->d_UF, (size_t)5 * m->nfpt * ts);
    if (!st) st = dalloc(m, &m->d_FV, (size_t)4 * m->nfpt * ts);
    // defined contents for the halo slots of a partitioned handle before its first exchange
    if (!st && m->nparts > 1 && (cudaMemset(m->d_UF, 0, (size_t)5 * m->nfpt * ts) != cudaSuccess ||
                                 cudaMemset(m->d_FV, 0, (size_t)4 * m->nfpt * ts) != cudaSuccess))
        st = fail(FR_ECUDA, "memset");
    if (!st) st = dalloc(m, (void **)&m->d_status, sizeof(int));
    if (!st && cudaMemset(m->d_status, 0, sizeof(int)) != cudaSuccess) st = fail(FR_ECUDA, "memset");
    if (!st && cudaMallocHost((void **)&m->h_status, sizeof(int)) != cudaSuccess) st = fail(FR_ENOMEM, "pinned status");
    if (!st && cudaEventCreateWithFlags(&m->ev_status, cudaEventDisableTiming) != cudaSuccess) st = fail(FR_ECUDA, "event");
    if (st) { fr_destroy(m); return st; }
    *m->h_status = 0;
    *out = m;
    return FR_OK;
}

extern "C" fr_status fr_destroy(fr_mesh *m)
{
    if (!m) return FR_OK;
    void **bufs[] = {&m->d_fnrm, (void **)&m->d_fnrm64, &m->d_geo64, (void **)&m->d_MF, (void **)&m->d_RL, &m->d_priops, &m->d_priops64, &m->d_tetops, &m->d_pyrops, &m->d_tetops64, &m->d_pyrops64, &m->d_geo, (void **)&m->d_partner, &m->d_UF, &m->d_FV, &m->d_CF, &m->d_QF, &m->d_DF, &m->d_Qu,
                     &m->d_UQ, &m->d_QQ, &m->d_Rt, &m->d_rk_k, &m->d_rk_us, (void **)&m->d_rk_acc, &m->d_io_U,
                     &m->d_io_R, (void **)&m->d_wsum, (void **)&m->d_status, &m->d_Qsnap, (void **)&m->d_qpartner,
                     &m->d_UFQ, &m->d_FVQ, (void **)&m->d_qlpts, &m->d_DQ, &m->d_mu, &m->d_mq, &m->d_mfn,
                     (void **)&m->d_send};
    for (void **b : bufs) dfree(*b);
    for (Group &g : m->groups) {
        dfree(g.d_geo); dfree((void *&)g.d_eu0); dfree((void *&)g.d_ef0); dfree((void *&)g.d_eph); dfree(g.d_phtab);
        dfree((void *&)g.d_lpts);
        dfree(g.d_geo64);
        dfree(g.d_fnrm);
        dfree((void *&)g.d_fnrm64);
    }
    if (m->h_status) cudaFreeHost(m->h_status);
    for (auto &t : m->timed) { cudaEventDestroy(t.a); cudaEventDestroy(t.b); }
    if (m->graph) cudaGraphExecDestroy(m->graph);
    for (auto e : m->ev_pool) cudaEventDestroy(e);
    if (m->ev_status) cudaEventDestroy(m->ev_status);
    delete m;
    return FR_OK;
}

extern "C" fr_status fr_set_debug(fr_mesh *m, int flags)
{
    if (!m) return fail(FR_EINVAL, "null handle");
    m->debug = flags;
    if (m->graph) { cudaGraphExecDestroy(m->graph); m->graph = nullptr; }   // recapture with the new arguments
    return FR_OK;
}

extern "C" fr_status fr_set_graph(fr_mesh *m, int on)
{
    if (!m) return fail(FR_EINVAL, "null handle");
    m->use_graph = on != 0;
    return FR_OK;
}

extern "C" fr_status fr_set_hex_tensor_cores(fr_mesh *m, int on)
{
    if (!m) return fail(FR_EINVAL, "null handle");
    m->hex_tc = on != 0;
    return FR_OK;
}

extern "C" fr_status fr_set_dense_tensor_cores(fr_mesh *m, int on)
{
    if (!m) return fail(FR_EINVAL, "null handle");
    m->dense_tc = on != 0;
    return FR_OK;
}

extern "C" fr_status fr_set_timing(fr_mesh *m, int on)
{
    if (!m) return fail(FR_EINVAL, "null handle");
    m->timing = on != 0;
    return FR_OK;
}

extern "C" fr_status fr_kernel_times(fr_mesh *m, double *ms, long long *count, int n_ids)
{
    if (!m || !ms || !count || n_ids <= 0) return fail(FR_EINVAL, "bad argument");
    for (int i = 0; i < n_ids; i++) { ms[i] = 0; count[i] = 0; }
    for (auto &t : m->timed) {
        CU(cudaEventSynchronize(t.b));
        float x = 0;
        CU(cudaEventElapsedTime(&x, t.a, t.b));
        if (t.kernel < n_ids) { ms[t.kernel] += x; count[t.kernel] += 1; }
        m->ev_pool.push_back(t.a);
        m->ev_pool.push_back(t.b);
    }
    m->timed.clear();
    return FR_OK;
}

extern "C" fr_status fr_set_form(fr_mesh *m, int form)
{
    if (!m || (form != FR_FUSED && form != FR_UNFUSED)) return fail(FR_EINVAL, "bad handle or form");
    m->form = form;
    return FR_OK;
}


// ---------------------------------------------------------------------------------------------
// Partitioned single mesh
//
// The fused RHS needs neighbour data at exactly two points, the boundaries of the paper's kernel
// groups (Sec. 2.2 and the kernel-grouping figure): the face solution U^(f) before con_u, and the
// face data of comm_flux (here the own-normal viscous flux, and in the low-Mach form the mass flux)
// before it. A mesh is split into nparts contiguous ranges of its global element order (hexahedra,
// then prisms, tetrahedra, pyramids; x fastest in the box meshes, so the ranges are z slabs). Each
// part owns its elements and flux points and holds, after them, one halo slot per remote partner
// point, peer by peer; the two exchanges fill the halo slots between the phases. Each side of a pair
// evaluates the common flux of its own point with the pair's global L/R roles, so a partitioned
// RHS equals the single-handle RHS bit for bit.
// ---------------------------------------------------------------------------------------------
struct PartPlan {
    long long E0 = 0, E1 = 0;              // own global elements [E0, E1)
    long long nfpt_own = 0;
    std::vector<long long> off;            // [nparts + 1]: first halo slot (and send entry) per peer
    std::vector<long long> send_g, recv_g; // full-mesh flux points sent / received, in buffer order
    std::vector<uint32_t> send_own;        // own flux index of every sent point
    std::vector<uint32_t> partner;         // partner codes of the own points (halo slots for remote ones)
};

static long long part_begin(long long ne, int nparts, int r) { return (long long)((__int128)ne * r / nparts); }

static fr_status part_plan(const fr_mesh *full, const std::vector<uint32_t> &pfull, int nparts, int part, PartPlan &pl)
{
    const long long ne = full->ne;
    pl.E0 = part_begin(ne, nparts, part);
    pl.E1 = part_begin(ne, nparts, part + 1);
    if (pl.E1 <= pl.E0) return fail(FR_EINVAL, "part %d of %d owns no element (%lld elements)", part, nparts, ne);
    auto rank_of = [&](long long ge) {
        int r = (int)((__int128)ge * nparts / ne);
        while (r + 1 < nparts && part_begin(ne, nparts, r + 1) <= ge) r++;
        while (r > 0 && part_begin(ne, nparts, r) > ge) r--;
        return r;
    };
    auto elem_of = [&](long long g) {
        for (const Block &B : full->blocks)
            if (g < B.f0 + B.ne * B.nf) return B.elem0 + (g - B.f0) / B.nf;
        return -1LL;
    };
    // own flux points in the restricted numbering: the own part of each block, in block order
    std::vector<long long> own_g;
    for (const Block &B : full->blocks) {
        const long long lo = std::max(B.elem0, pl.E0), hi = std::min(B.elem0 + B.ne, pl.E1);
        for (long long g = B.f0 + (lo - B.elem0) * B.nf; hi > lo && g < B.f0 + (hi - B.elem0) * B.nf; g++) own_g.push_back(g);
    }
    pl.nfpt_own = (long long)own_g.size();
    std::unordered_map<long long, uint32_t> own_idx;
    own_idx.reserve(own_g.size() * 2);
    for (size_t i = 0; i < own_g.size(); i++) own_idx[own_g[i]] = (uint32_t)i;
    struct Remote { int rank; long long pg; uint32_t own; };
    std::vector<Remote> rem;
    pl.partner.assign(own_g.size(), 0u);
    for (size_t i = 0; i < own_g.size(); i++) {
        const uint32_t pc = pfull[(size_t)own_g[i]];
        const long long pg = pc & ~FR_LFLAG;
        auto it = own_idx.find(pg);
        if (it != own_idx.end()) pl.partner[i] = it->second | (pc & FR_LFLAG);
        else rem.push_back(Remote{rank_of(elem_of(pg)), pg, (uint32_t)i});
    }
    if (pl.nfpt_own + (long long)rem.size() >= (long long)FR_LFLAG) return fail(FR_EUNSUPPORTED, "more than 2^31 flux points");
    pl.off.assign((size_t)nparts + 1, 0);
    for (const Remote &r : rem) pl.off[(size_t)r.rank + 1]++;
    for (int q = 0; q < nparts; q++) pl.off[(size_t)q + 1] += pl.off[(size_t)q];
    // halo slots of peer q sorted by the remote point's full index; the matching send list of this
    // part for q is its own points whose partner lies on q, sorted by their own full index: both
    // sides order the same pairs the same way
    std::vector<Remote> by_pg = rem, by_g = rem;
    std::sort(by_pg.begin(), by_pg.end(), [](const Remote &a, const Remote &b) { return a.rank != b.rank ? a.rank < b.rank : a.pg < b.pg; });
    std::sort(by_g.begin(), by_g.end(), [&](const Remote &a, const Remote &b) { return a.rank != b.rank ? a.rank < b.rank : own_g[a.own] < own_g[b.own]; });
    pl.recv_g.resize(rem.size()); pl.send_g.resize(rem.size()); pl.send_own.resize(rem.size());
    for (size_t k = 0; k < rem.size(); k++) {
        const Remote &r = by_pg[k];
        pl.recv_g[k] = r.pg;
        pl.partner[r.own] = (uint32_t)(pl.nfpt_own + (long long)k) | (pfull[(size_t)own_g[r.own]] & FR_LFLAG);
        pl.send_g[k] = own_g[by_g[k].own];
        pl.send_own[k] = by_g[k].own;
    }
    return FR_OK;
}

// Host-only: the exchange plan of one part, with nothing built on the device.
extern "C" fr_status fr_partition_plan(const fr_mesh_desc *desc, const fr_params *prm, int nparts, int part,
                                       long long *info, long long *counts, long long *send_g, long long *recv_g,
                                       long long cap)
{
    if (!desc || !prm || !info || nparts < 1 || part < 0 || part >= nparts) return fail(FR_EINVAL, "bad argument");
    fr_mesh full;
    std::vector<uint32_t> pfull;
    fr_status st = build_host(&full, &desc, 1, prm, pfull);
    if (st) return st;
    if (full.surf) return fail(FR_EUNSUPPORTED, "partitioned meshes run without surface-flux anti-aliasing");
    PartPlan pl;
    st = part_plan(&full, pfull, nparts, part, pl);
    if (st) return st;
    const long long n = (long long)pl.recv_g.size();
    info[0] = pl.E0; info[1] = pl.E1; info[2] = pl.nfpt_own; info[3] = n; info[4] = full.ne; info[5] = full.nfpt;
    if (counts)
        for (int q = 0; q < nparts; q++) counts[q] = pl.off[(size_t)q + 1] - pl.off[(size_t)q];
    if ((send_g || recv_g) && cap < n) return fail(FR_EINVAL, "plan buffers hold %lld entries, %lld needed", cap, n);
    for (long long k = 0; k < n; k++) {
        if (send_g) send_g[k] = pl.send_g[(size_t)k];
        if (recv_g) recv_g[k] = pl.recv_g[(size_t)k];
    }
    return FR_OK;
}

extern "C" fr_status fr_mesh_create_part(const fr_mesh_desc *desc, const fr_params *prm, int nparts, int part, fr_mesh **out)
{
    if (!out) return fail(FR_EINVAL, "out is null");
    *out = nullptr;
    if (!desc || !prm || nparts < 1 || part < 0 || part >= nparts) return fail(FR_EINVAL, "bad argument");
    fr_mesh full;
    std::vector<uint32_t> pfull;
    fr_status st = build_host(&full, &desc, 1, prm, pfull);
    if (st) return st;
    if (full.surf) return fail(FR_EUNSUPPORTED, "partitioned meshes run without surface-flux anti-aliasing");
    PartPlan pl;
    st = part_plan(&full, pfull, nparts, part, pl);
    if (st) return st;
    fr_mesh *m = new fr_mesh();
    m->nparts = nparts; m->part = part; m->E0 = pl.E0; m->E1 = pl.E1; m->nfpt_own = pl.nfpt_own;
    m->halo_off = pl.off;
    m->prec = full.prec; m->curved = full.curved;
    m->pri = full.pri; m->has_pri = full.has_pri;
    m->tet = full.tet; m->has_tet = full.has_tet;
    m->pyr = full.pyr; m->has_pyr = full.has_pyr;
    // the own elements of the single instance, block by block, with their geometry
    const InstanceHost &F = full.inst[0];
    InstanceHost I;
    I.prm = F.prm;
    I.n_hex = I.n_pri = I.n_tet = I.n_pyr = 0;
    long long elem = 0, u = 0, f = 0;
    for (size_t b = 0; b < full.blocks.size(); b++) {
        const Block &B = full.blocks[b];
        const long long lo = std::max(B.elem0, pl.E0), hi = std::min(B.elem0 + B.ne, pl.E1);
        if (hi <= lo) continue;
        Block nb = B;
        nb.ne = hi - lo; nb.elem0 = elem; nb.u0 = u; nb.f0 = f;
        (B.type == 0 ? I.n_hex : B.type == 1 ? I.n_pri : B.type == 2 ? I.n_tet : I.n_pyr) += (int)nb.ne;
        for (long long ge = lo; ge < hi; ge++) {   // single instance: instance-local index = global index
            I.x0J.insert(I.x0J.end(), F.x0J.begin() + ge * 12, F.x0J.begin() + ge * 12 + 12);
            I.curved.push_back(F.curved[(size_t)ge]);
            I.vx.insert(I.vx.end(), F.vx.begin() + ge * 24, F.vx.begin() + ge * 24 + 24);
            m->geo_host.insert(m->geo_host.end(), full.geo_host.begin() + ge * 10, full.geo_host.begin() + ge * 10 + 10);
        }
        m->blocks.push_back(nb);
        m->hex1d.push_back(full.hex1d[b]);
        elem += nb.ne; u += nb.ne * FR_NV * nb.nu; f += nb.ne * nb.nf;
    }
    m->inst.push_back(I);
    m->ne = elem; m->nU = u;
    m->nfpt = f + (pl.off.back());
    m->inst_u0 = {0, u};
    if (f != pl.nfpt_own) { delete m; return fail(FR_EMESH, "partition bookkeeping mismatch"); }
    st = finish_create(m, pl.partner, out);
    if (st) return st;
    m = *out;
    if (!pl.send_own.empty()) {
        st = dalloc(m, (void **)&m->d_send, pl.send_own.size() * sizeof(uint32_t));
        if (!st && cudaMemcpy(m->d_send, pl.send_own.data(), pl.send_own.size() * sizeof(uint32_t), cudaMemcpyHostToDevice) != cudaSuccess)
            st = fail(FR_ECUDA, "send list upload failed");
        if (st) { fr_destroy(m); *out = nullptr; return st; }
    }
    return FR_OK;
}

extern "C" fr_status fr_halo_info(const fr_mesh *m, long long *info, long long *counts)
{
    if (!m || !info) return fail(FR_EINVAL, "null argument");
    info[0] = m->nparts; info[1] = m->part; info[2] = m->E0; info[3] = m->E1;
    info[4] = m->nfpt - m->nfpt_own;
    info[5] = FR_NV;                                                    // values per point, exchange 0
    info[6] = 4 + ((m->prec != FR_FP64 && m->lowmach) ? 2 : 0);         // values per point, exchange 1
    if (counts)
        for (int q = 0; q < m->nparts; q++)
            counts[q] = m->halo_off.empty() ? 0 : m->halo_off[(size_t)q + 1] - m->halo_off[(size_t)q];
    return FR_OK;
}

// Halo buffers: peer by peer (increasing rank), a segment of nvar x count values, var-major.
// what = 0: the face solution (5 values); what = 1: the own-normal viscous flux (4 values) and, in
// the low-Mach form, the float-float mass flux (2 floats).
template <typename T>
__global__ void k_halo_pack(const T *UF, const T *FV, const ff *MF, long long nfpt, int what, int nvar,
                            const uint32_t *idx, long long n, T *buf)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvar * n; i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(i / n);
        const long long g = idx[i % n];
        T val;
        if (what == 0) val = UF[v * nfpt + g];
        else if (v < 4) val = FV[v * nfpt + g];
        else val = (T)(v == 4 ? MF[g].hi : MF[g].lo);
        buf[i] = val;
    }
}

template <typename T>
__global__ void k_halo_unpack(T *UF, T *FV, ff *MF, long long nfpt, int what, int nvar, long long slot0, long long n,
                              const T *buf)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nvar * n; i += (long long)gridDim.x * blockDim.x) {
        const int v = (int)(i / n);
        const long long g = slot0 + i % n;
        const T val = buf[i];
        if (what == 0) UF[v * nfpt + g] = val;
        else if (v < 4) FV[v * nfpt + g] = val;
        else if (v == 4) MF[g].hi = (float)val;
        else MF[g].lo = (float)val;
    }
}

template <typename T>
static fr_status halo_impl(fr_mesh *m, int what, void *buf, bool pack, cudaStream_t s)
{
    long long info[7];
    fr_halo_info(m, info, nullptr);
    const int nvar = (int)info[5 + what];
    for (int q = 0; q < m->nparts; q++) {
        const long long o = m->halo_off[(size_t)q], n = m->halo_off[(size_t)q + 1] - o;
        if (n == 0) continue;
        T *seg = reinterpret_cast<T *>(buf) + nvar * o;
        const int grid = (int)std::min<long long>((nvar * n + 255) / 256, 8LL * m->nsm);
        if (pack)
            k_halo_pack<T><<<grid, 256, 0, s>>>(reinterpret_cast<const T *>(m->d_UF), reinterpret_cast<const T *>(m->d_FV),
                                                reinterpret_cast<const ff *>(m->d_MF), m->nfpt, what, nvar, m->d_send + o, n, seg);
        else
            k_halo_unpack<T><<<grid, 256, 0, s>>>(reinterpret_cast<T *>(m->d_UF), reinterpret_cast<T *>(m->d_FV),
                                                  reinterpret_cast<ff *>(m->d_MF), m->nfpt, what, nvar, m->nfpt_own + o, n, seg);
        CU(cudaPeekAtLastError());
    }
    return FR_OK;
}

extern "C" fr_status fr_halo_pack(fr_mesh *m, int what, void *send_dev, void *stream)
{
    if (!m || (what != 0 && what != 1)) return fail(FR_EINVAL, "bad argument");
    if (m->nfpt == m->nfpt_own) return FR_OK;
    if (!send_dev) return fail(FR_EINVAL, "null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    return m->prec == FR_FP64 ? halo_impl<double>(m, what, send_dev, true, s) : halo_impl<float>(m, what, send_dev, true, s);
}

extern "C" fr_status fr_halo_unpack(fr_mesh *m, int what, const void *recv_dev, void *stream)
{
    if (!m || (what != 0 && what != 1)) return fail(FR_EINVAL, "bad argument");
    if (m->nfpt == m->nfpt_own) return FR_OK;
    if (!recv_dev) return fail(FR_EINVAL, "null buffer");
    cudaStream_t s = (cudaStream_t)stream;
    return m->prec == FR_FP64 ? halo_impl<double>(m, what, const_cast<void *>(recv_dev), false, s)
                              : halo_impl<float>(m, what, const_cast<void *>(recv_dev), false, s);
}

// ---------------------------------------------------------------------------------------------
// RHS
// ---------------------------------------------------------------------------------------------
template <typename T>
static HexArgs<T> make_args(fr_mesh *m, const Block &b, const void *U, void *R)
{
    HexArgs<T> a{};
    const InstanceHost &I = m->inst[b.inst];
    a.ne = b.ne; a.u0 = b.u0; a.f0 = b.f0; a.nfpt = m->nfpt;
    a.geo = reinterpret_cast<const Geo<T> *>(m->d_geo) + b.elem0;
    a.partner = m->d_partner;
    a.ph = phys_of<T>(I.prm);
    a.ph.dev = m->lowmach ? 1 : 0;
    a.geo64 = m->d_geo64 ? reinterpret_cast<const GeoLM *>(m->d_geo64) + b.elem0 : nullptr;
    a.MF = reinterpret_cast<ff *>(m->d_MF);
    a.RL = reinterpret_cast<ff *>(m->d_RL);
    a.fnrm = m->d_fnrm ? reinterpret_cast<const T *>(m->d_fnrm) + b.elem0 * 24 : nullptr;
    a.fnrm64 = m->d_fnrm64 ? reinterpret_cast<const ff *>(m->d_fnrm64) + b.elem0 * 24 : nullptr;
    a.U = reinterpret_cast<const T *>(U); a.R = reinterpret_cast<T *>(R);
    a.UF = reinterpret_cast<T *>(m->d_UF); a.FV = reinterpret_cast<T *>(m->d_FV);
    a.CF = reinterpret_cast<T *>(m->d_CF); a.QF = reinterpret_cast<T *>(m->d_QF); a.DF = reinterpret_cast<T *>(m->d_DF);
    // per-element unfused arrays are addressed block-locally; the unfused form runs single-block meshes
    a.Qu = reinterpret_cast<T *>(m->d_Qu); a.UQ = reinterpret_cast<T *>(m->d_UQ); a.QQ = reinterpret_cast<T *>(m->d_QQ);
    a.Rt = reinterpret_cast<T *>(m->d_Rt);
    a.status = m->d_status;
    a.dbg_wait0 = (m->debug & 2) ? 1 : 0;
    a.nU = m->nU;
    a.tcmode = m->prec == FR_MIXED_FP16 ? 1 : (m->prec == FR_MIXED_BF16 ? 2 : 0);
    if (b.type == 0 && !m->hex_tc) a.tcmode = 0;
    if ((b.type == 2 || b.type == 3) && !m->dense_tc) a.tcmode = 0;
    a.aa_off = b.m == b.p + 1;
    if (a.aa_off) a.tcmode = 0;
    if (m->surf) {
        a.surf = 1;
        a.qpartner = m->d_qpartner;
        a.UFQ = reinterpret_cast<T *>(m->d_UFQ);
        a.FVQ = reinterpret_cast<T *>(m->d_FVQ);
        a.DQ = reinterpret_cast<T *>(m->d_DQ);
        a.qlpts = m->d_qlpts;
        a.nqf = m->nqf;
        a.nqlpts = m->nqlpts;
        a.tcmode = 0;
    }
    if (m->curved) {
        a.tcmode = 0;   // the tensor-core volume kernels keep an element-constant metric
        a.mu = reinterpret_cast<const T *>(m->d_mu);
        a.mq = reinterpret_cast<const T *>(m->d_mq);
        a.mfn = reinterpret_cast<const T *>(m->d_mfn);
    }
    return a;
}

static fr_status ensure_unfused(fr_mesh *m)
{
    if (m->blocks.size() != 1 || m->blocks[0].type != 0)
        return fail(FR_EUNSUPPORTED, "the unfused form runs single-instance hexahedral meshes");
    if (m->blocks[0].m != m->blocks[0].p + 2 || m->surf)
        return fail(FR_EUNSUPPORTED, "the unfused form runs the flux-anti-aliased discretisation only");
    const Block &b = m->blocks[0];
    size_t ts = tsize(m->prec);
    long long nq = (long long)b.m * b.m * b.m;
    fr_status st = FR_OK;
    if (!st) st = dalloc(m, &m->d_CF, (size_t)5 * m->nfpt * ts);
    if (!st) st = dalloc(m, &m->d_QF, (size_t)15 * m->nfpt * ts);
    if (!st) st = dalloc(m, &m->d_DF, (size_t)5 * m->nfpt * ts);
    if (!st) st = dalloc(m, &m->d_Qu, (size_t)15 * b.ne * b.nu * ts);
    if (!st) st = dalloc(m, &m->d_UQ, (size_t)5 * b.ne * nq * ts);
    if (!st) st = dalloc(m, &m->d_QQ, (size_t)15 * b.ne * nq * ts);
    if (!st) st = dalloc(m, &m->d_Rt, (size_t)5 * b.ne * b.nu * ts);
    return st;
}

static fr_status status_error(int v)
{
    if (v & 4) return fail(FR_EBOUNDS, "an index check of the bounds-checking build failed on the device");
    if (v & 2) return fail(FR_ETIMEOUT, "a bounded tensor-core completion wait gave up on the device");
    return fail(FR_ENONPHYS, "non-physical state met on the device");
}

static fr_status check_status(fr_mesh *m)
{
    if (m->status_pending && cudaEventQuery(m->ev_status) == cudaSuccess) {
        m->status_pending = false;
        if (*m->h_status) {
            const int v = *m->h_status;
            *m->h_status = 0;
            cudaMemset(m->d_status, 0, sizeof(int));
            return status_error(v);
        }
    }
    return FR_OK;
}

static fr_status post_status(fr_mesh *m, cudaStream_t s)
{
    CU(cudaMemcpyAsync(m->h_status, m->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CU(cudaEventRecord(m->ev_status, s));
    m->status_pending = true;
    return FR_OK;
}

// The groups can share one launch per phase: two to FR_MULTI_MAX groups of hexahedra (p = 3 or 4)
// and prisms with flux anti-aliasing on the CUDA cores (no tensor-core split products, no surface-flux
// anti-aliasing, affine elements).
static bool can_merge(const fr_mesh *m)
{
    if (m->form != FR_FUSED || m->surf || m->curved || m->groups.size() < 2 || m->groups.size() > FR_MULTI_MAX)
        return false;
    for (const Group &g : m->groups) {
        const Block &b = m->blocks[g.blks[0]];
        if (b.m != b.p + 2) return false;
        if (b.type == 0 && (b.p < 3 || b.p > 4 || (m->prec >= FR_MIXED_BF16 && m->hex_tc))) return false;
        if (b.type == 1 && m->prec >= FR_MIXED_BF16) return false;   // the mixed forms' prisms use the tensor cores
        if (b.type > 1) return false;
    }
    return true;
}

// RK4 stage folded into the fused interface kernel (stage < 0: plain RHS).
struct RkFold {
    int stage = -1;
    double dt = 0;
    double *U = nullptr, *acc = nullptr;
    void *us = nullptr;
};

// only >= 0: just that phase of the fused form (0 face solution, 1 volume group, 2 interface group).
template <typename T>
static fr_status rhs_impl(fr_mesh *m, const void *U, void *R, cudaStream_t s, const RkFold &rk = RkFold(), int only = -1)
{
    if (m->nparts > 1 && (m->form != FR_FUSED || only < 0))
        return fail(FR_EUNSUPPORTED, "a partitioned mesh runs the fused phases one at a time (fr_rhs_phase) with "
                                     "halo exchanges between them");
    if (m->form == FR_FUSED && m->merged && can_merge(m)) {
        // one launch per phase over every group (each side evaluates its own points' common flux)
        for (int ph = 0; ph < 3; ph++) {
            if (only >= 0 && ph != only) continue;
            TimeScope ts(m, ph, s);
            MultiArgs<T> ma{};
            ma.ng = (int)m->groups.size();
            ma.pops = reinterpret_cast<const PriOps<T> *>(m->d_priops);
            ma.pff = reinterpret_cast<const PriOpsFF *>(m->d_priops64);
            for (int gi = 0; gi < ma.ng; gi++) {
                const Group &gr = m->groups[(size_t)gi];
                const Block &b = m->blocks[gr.blks[0]];
                HexArgs<T> a = make_args<T>(m, b, U, R);
                if (gr.blks.size() > 1) {
                    a.ne = gr.ne; a.u0 = 0; a.f0 = 0;
                    a.geo = reinterpret_cast<const Geo<T> *>(gr.d_geo);
                    a.eu0 = gr.d_eu0; a.ef0 = gr.d_ef0; a.eph = gr.d_eph;
                    if (m->lowmach) a.geo64 = reinterpret_cast<const GeoLM *>(gr.d_geo64);
                    a.fnrm = reinterpret_cast<const T *>(gr.d_fnrm);
                    a.fnrm64 = reinterpret_cast<const ff *>(gr.d_fnrm64);
                    a.phtab = reinterpret_cast<const Phys<T> *>(gr.d_phtab);
                }
                a.tcmode = 0;
                if (ph == 2 && rk.stage >= 0) {
                    a.rkstage = rk.stage + 1; a.rkdt = rk.dt; a.rkU = rk.U; a.rkacc = rk.acc;
                    a.rkus = reinterpret_cast<T *>(rk.us);
                }
                ma.kind[gi] = b.type == 1 ? 1 : b.p;
                ma.a[gi] = a;
            }
            if (multi_phase<T>(ph, ma, s)) return fail(FR_ECUDA, "merged phase %d launch: %s", ph, cudaGetErrorString(cudaGetLastError()));
        }
    } else if (m->form == FR_FUSED) {
        static const int plain[3] = {0, 1, 2}, split[4] = {0, 1, 3, 4};
        const int *phases = m->split_c ? split : plain;
        int nph = m->split_c ? 4 : 3;
        if (only >= 0) {   // one phase: 0 -> A, 1 -> B, 2 -> C (or C1 + C2)
            phases += only;
            nph = only < 2 ? 1 : nph - 2;
        }
        for (int pi = 0; pi < nph; pi++) {
            const int ph = phases[pi];
            TimeScope ts(m, ph, s);
            for (const Group &gr : m->groups) {
                const Block &b = m->blocks[gr.blks[0]];
                HexArgs<T> a = make_args<T>(m, b, U, R);
                if (gr.blks.size() > 1) {
                    a.ne = gr.ne; a.u0 = 0; a.f0 = 0;
                    a.geo = reinterpret_cast<const Geo<T> *>(gr.d_geo);
                    a.eu0 = gr.d_eu0; a.ef0 = gr.d_ef0; a.eph = gr.d_eph;
                    if (m->lowmach) a.geo64 = reinterpret_cast<const GeoLM *>(gr.d_geo64);
                    a.fnrm = reinterpret_cast<const T *>(gr.d_fnrm);
                    a.fnrm64 = reinterpret_cast<const ff *>(gr.d_fnrm64);
                    a.phtab = reinterpret_cast<const Phys<T> *>(gr.d_phtab);
                }
                a.lpts = gr.d_lpts; a.nlpts = gr.nlpts;
                if ((ph == 2 || ph == 4) && rk.stage >= 0) {
                    a.rkstage = rk.stage + 1; a.rkdt = rk.dt; a.rkU = rk.U; a.rkacc = rk.acc;
                    a.rkus = reinterpret_cast<T *>(rk.us);
                }
                int lr = b.type == 0 ? hex_fused_phase<T>(b.p, ph, a, s, gr.variant)
                         : b.type == 1 ? pri_fused_phase<T>(ph, a, reinterpret_cast<const PriOps<T> *>(m->d_priops), reinterpret_cast<const PriOpsFF *>(m->d_priops64), s)
                         : b.type == 2 ? tet_fused_phase<T>(ph, a, reinterpret_cast<const TetOps<T> *>(m->d_tetops), reinterpret_cast<const DenseOpsFF<TetOps<float>> *>(m->d_tetops64), s)
                                       : pyr_fused_phase<T>(ph, a, reinterpret_cast<const PyrOps<T> *>(m->d_pyrops), reinterpret_cast<const DenseOpsFF<PyrOps<float>> *>(m->d_pyrops64), s);
                if (lr) return fail(FR_ECUDA, "fused phase %d launch: %s", ph, cudaGetErrorString(cudaGetLastError()));
            }
        }
    } else {
        fr_status st = ensure_unfused(m);
        if (st) return st;
        const Block &b = m->blocks[0];
        HexArgs<T> a = make_args<T>(m, b, U, R);
        a.ph.dev = 0;   // the unfused form is the plain one-kernel-per-stage form
        for (int k = 1; k <= 13; k++) {
            int lr;
            {
                TimeScope ts(m, 10 + k, s);
                lr = hex_unfused_kernel<T>(b.p, k, a, s);
            }
            if (lr) return fail(FR_ECUDA, "unfused kernel %d launch: %s", k, cudaGetErrorString(cudaGetLastError()));
            if (k == 6 && m->debug) {
                size_t bytes = (size_t)15 * b.ne * b.nu * sizeof(T);
                st = dalloc(m, &m->d_Qsnap, bytes);
                if (st) return st;
                CU(cudaMemcpyAsync(m->d_Qsnap, m->d_Qu, bytes, cudaMemcpyDeviceToDevice, s));
            }
        }
    }
    return FR_OK;
}

static fr_status rhs_dispatch(fr_mesh *m, const void *U, void *R, cudaStream_t s)
{
    return m->prec == FR_FP64 ? rhs_impl<double>(m, U, R, s) : rhs_impl<float>(m, U, R, s);
}

extern "C" fr_status fr_rhs_phase(fr_mesh *m, int phase, const void *U_dev, void *R_dev, void *stream)
{
    if (!m || !U_dev || !R_dev || phase < 0 || phase > 2) return fail(FR_EINVAL, "bad argument");
    if (U_dev == R_dev) return fail(FR_EINVAL, "U and R must not alias");
    if (m->form != FR_FUSED) return fail(FR_EUNSUPPORTED, "fr_rhs_phase runs the fused form");
    fr_status st = check_status(m);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = m->prec == FR_FP64 ? rhs_impl<double>(m, U_dev, R_dev, s, RkFold(), phase)
                            : rhs_impl<float>(m, U_dev, R_dev, s, RkFold(), phase);
    if (st) return st;
    return phase == 2 ? post_status(m, s) : FR_OK;
}

// Launch shapes of a hexahedral group's volume kernel: 0, 1, 2 = one element per CTA of 64, 128,
// 256 threads; FP32 p = 3 with flux anti-aliasing on the CUDA cores also 3, 4 = eight elements per
// CTA with register-resident line sweeps (one or two CTAs per SM).
static int volume_shapes(const fr_mesh *m, const Block &b)
{
    const bool b32 = m->prec != FR_FP64 && b.p == 3 && b.m == b.p + 2 && !m->surf && !m->curved &&
                     (m->prec == FR_FP32 || !m->hex_tc);
    return b32 ? 6 : 3;
}

extern "C" fr_status fr_set_merged(fr_mesh *m, int on)
{
    if (!m) return fail(FR_EINVAL, "null handle");
    if (on && !can_merge(m))
        return fail(FR_EUNSUPPORTED, "one launch per phase needs 2 to %d groups of hexahedra (p = 3, 4) and prisms "
                                     "on the CUDA cores, flux anti-aliasing, affine elements", FR_MULTI_MAX);
    m->merged = on != 0;
    if (m->graph) { cudaGraphExecDestroy(m->graph); m->graph = nullptr; }
    return FR_OK;
}

extern "C" fr_status fr_set_rk_fp64_stages(fr_mesh *m, int on)
{
    if (!m) return fail(FR_EINVAL, "null handle");
    m->rk_wide = on != 0;
    if (m->graph) { cudaGraphExecDestroy(m->graph); m->graph = nullptr; }
    return FR_OK;
}

extern "C" fr_status fr_set_volume_shape(fr_mesh *m, int shape)
{
    if (!m || shape < 0 || shape > 5) return fail(FR_EINVAL, "bad argument");
    for (Group &g : m->groups) {
        const Block &b = m->blocks[g.blks[0]];
        if (b.type != 0) continue;
        if (shape >= volume_shapes(m, b))
            return fail(FR_EUNSUPPORTED, "volume-kernel shape %d needs FP32, p = 3, flux anti-aliasing, affine elements", shape);
    }
    for (Group &g : m->groups)
        if (m->blocks[g.blks[0]].type == 0) g.variant = shape;
    if (m->graph) { cudaGraphExecDestroy(m->graph); m->graph = nullptr; }
    return FR_OK;
}

extern "C" fr_status fr_group_info(const fr_mesh *m, int group, long long *info)
{
    if (!m || !info) return fail(FR_EINVAL, "null argument");
    if (group < 0 || group >= (int)m->groups.size()) return fail(FR_EINVAL, "group %d of %d", group, (int)m->groups.size());
    const Group &g = m->groups[(size_t)group];
    const Block &b = m->blocks[g.blks[0]];
    info[0] = b.type; info[1] = b.p; info[2] = b.m; info[3] = g.ne; info[4] = g.variant;
    info[5] = b.type == 0 ? volume_shapes(m, b) : 1;
    return FR_OK;
}

extern "C" fr_status fr_set_group_shape(fr_mesh *m, int group, int shape)
{
    if (!m) return fail(FR_EINVAL, "null handle");
    if (group < 0 || group >= (int)m->groups.size()) return fail(FR_EINVAL, "group %d of %d", group, (int)m->groups.size());
    Group &g = m->groups[(size_t)group];
    const Block &b = m->blocks[g.blks[0]];
    if (b.type != 0 || shape < 0 || shape >= volume_shapes(m, b))
        return fail(FR_EUNSUPPORTED, "group %d has no volume-kernel shape %d", group, shape);
    g.variant = shape;
    if (m->graph) { cudaGraphExecDestroy(m->graph); m->graph = nullptr; }
    return FR_OK;
}

// Times every launch shape of the volume kernel of each hexahedral group on the caller's state and
// keeps the fastest. Every shape computes each output with the same operations, so results do not
// depend on the choice.
template <typename T>
static fr_status autotune_impl(fr_mesh *m, const void *U, void *R, cudaStream_t s, int *chosen)
{
    if (m->curved) {   // the fused volume kernels (the ones tuned) do not run curved meshes
        for (size_t gi = 0; gi < m->groups.size(); gi++) chosen[gi] = m->groups[gi].variant;
        return FR_OK;
    }
    // face solution of the current state first (the volume kernel reads it)
    for (const Group &gr : m->groups) {
        const Block &b = m->blocks[gr.blks[0]];
        HexArgs<T> a = make_args<T>(m, b, U, R);
        if (gr.blks.size() > 1) {
            a.ne = gr.ne; a.u0 = 0; a.f0 = 0;
            a.geo = reinterpret_cast<const Geo<T> *>(gr.d_geo);
            a.eu0 = gr.d_eu0; a.ef0 = gr.d_ef0; a.eph = gr.d_eph;
            a.phtab = reinterpret_cast<const Phys<T> *>(gr.d_phtab);
            if (m->lowmach) a.geo64 = reinterpret_cast<const GeoLM *>(gr.d_geo64);
            a.fnrm = reinterpret_cast<const T *>(gr.d_fnrm);
            a.fnrm64 = reinterpret_cast<const ff *>(gr.d_fnrm64);
        }
        int lr = b.type == 0 ? hex_fused_phase<T>(b.p, 0, a, s, gr.variant)
                 : b.type == 1 ? pri_fused_phase<T>(0, a, reinterpret_cast<const PriOps<T> *>(m->d_priops), reinterpret_cast<const PriOpsFF *>(m->d_priops64), s)
                 : b.type == 2 ? tet_fused_phase<T>(0, a, reinterpret_cast<const TetOps<T> *>(m->d_tetops), reinterpret_cast<const DenseOpsFF<TetOps<float>> *>(m->d_tetops64), s)
                               : pyr_fused_phase<T>(0, a, reinterpret_cast<const PyrOps<T> *>(m->d_pyrops), reinterpret_cast<const DenseOpsFF<PyrOps<float>> *>(m->d_pyrops64), s);
        if (lr) return fail(FR_ECUDA, "autotune: face phase launch failed");
    }
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    CU(cudaEventCreate(&e1));
    int gi = 0;
    for (Group &gr : m->groups) {
        const Block &b = m->blocks[gr.blks[0]];
        if (b.type != 0) { chosen[gi++] = gr.variant; continue; }
        HexArgs<T> a = make_args<T>(m, b, U, R);
        if (gr.blks.size() > 1) {
            a.ne = gr.ne; a.u0 = 0; a.f0 = 0;
            a.geo = reinterpret_cast<const Geo<T> *>(gr.d_geo);
            a.eu0 = gr.d_eu0; a.ef0 = gr.d_ef0; a.eph = gr.d_eph;
            a.phtab = reinterpret_cast<const Phys<T> *>(gr.d_phtab);
            if (m->lowmach) a.geo64 = reinterpret_cast<const GeoLM *>(gr.d_geo64);
            a.fnrm = reinterpret_cast<const T *>(gr.d_fnrm);
            a.fnrm64 = reinterpret_cast<const ff *>(gr.d_fnrm64);
        }
        float best = 1e30f;
        int bestv = gr.variant;
        for (int v = 0; v < volume_shapes(m, b); v++) {
            if (hex_fused_phase<T>(b.p, 1, a, s, v)) return fail(FR_ECUDA, "autotune: volume launch failed");  // warm-up
            CU(cudaEventRecord(e0, s));
            for (int r = 0; r < 2; r++) hex_fused_phase<T>(b.p, 1, a, s, v);
            CU(cudaEventRecord(e1, s));
            CU(cudaEventSynchronize(e1));
            float ms = 0;
            CU(cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) { best = ms; bestv = v; }
        }
        gr.variant = bestv;
        chosen[gi++] = bestv;
    }
    if (can_merge(m)) {
        // whole RHS with per-group launches against one launch per phase over all groups
        float t[2] = {0.f, 0.f};
        for (int mg = 0; mg < 2; mg++) {
            m->merged = mg;
            fr_status r = rhs_impl<T>(m, U, R, s);   // warm-up
            if (r) { cudaEventDestroy(e0); cudaEventDestroy(e1); return r; }
            CU(cudaEventRecord(e0, s));
            for (int rep = 0; rep < 3; rep++) rhs_impl<T>(m, U, R, s);
            CU(cudaEventRecord(e1, s));
            CU(cudaEventSynchronize(e1));
            CU(cudaEventElapsedTime(&t[mg], e0, e1));
        }
        m->merged = t[1] < t[0];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CU(cudaPeekAtLastError());
    if (m->graph) { cudaGraphExecDestroy(m->graph); m->graph = nullptr; }   // recapture with the new shapes
    return FR_OK;
}

extern "C" fr_status fr_autotune(fr_mesh *m, const void *U_dev, void *R_dev, int *chosen, int n_chosen, void *stream)
{
    if (!m || !U_dev || !R_dev) return fail(FR_EINVAL, "null argument");
    std::vector<int> tmp(m->groups.size(), 0);
    fr_status st = m->prec == FR_FP64 ? autotune_impl<double>(m, U_dev, R_dev, (cudaStream_t)stream, tmp.data())
                                      : autotune_impl<float>(m, U_dev, R_dev, (cudaStream_t)stream, tmp.data());
    if (st) return st;
    if (chosen)
        for (int i = 0; i < n_chosen && i < (int)tmp.size(); i++) chosen[i] = tmp[i];
    return check_status(m);
}

extern "C" fr_status fr_rhs(fr_mesh *m, const void *U_dev, void *R_dev, void *stream)
{
    if (!m || !U_dev || !R_dev) return fail(FR_EINVAL, "null argument");
    if (U_dev == R_dev) return fail(FR_EINVAL, "U and R must not alias");
    fr_status st = check_status(m);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = rhs_dispatch(m, U_dev, R_dev, s);
    if (st) return st;
    return post_status(m, s);
}

extern "C" fr_status fr_rhs_host(fr_mesh *m, const void *U_host, void *R_host, void *stream)
{
    if (!m || !U_host || !R_host) return fail(FR_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = (size_t)m->nU * tsize(m->prec);
    fr_status st = dalloc(m, &m->d_io_U, (size_t)m->nU * sizeof(double));
    if (!st) st = dalloc(m, &m->d_io_R, bytes);
    if (st) return st;
    CU(cudaMemcpyAsync(m->d_io_U, U_host, bytes, cudaMemcpyHostToDevice, s));
    st = fr_rhs(m, m->d_io_U, m->d_io_R, stream);
    if (st) return st;
    CU(cudaMemcpyAsync(R_host, m->d_io_R, bytes, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return check_status(m);
}

extern "C" fr_status fr_sync_status(fr_mesh *m, void *stream)
{
    if (!m) return fail(FR_EINVAL, "null handle");
    CU(cudaStreamSynchronize((cudaStream_t)stream));
    int v = 0;
    CU(cudaMemcpy(&v, m->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    CU(cudaMemset(m->d_status, 0, sizeof(int)));
    m->status_pending = false;
    *m->h_status = 0;
    return v ? status_error(v) : FR_OK;
}

// ---------------------------------------------------------------------------------------------
// RK4
// ---------------------------------------------------------------------------------------------
// FP64 unfused form, after stage s (k = R(u_s)): acc (+)= b_s k; u_{s+1} = U + c_{s+1} dt k; the last
// stage updates U.
__global__ void k_rk_update64(double *__restrict__ U, const double *__restrict__ k, double *__restrict__ acc,
                              double *__restrict__ us, long long n, double dt, int stage)
{
    const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const double cnext[4] = {0.5, 0.5, 1.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double kv = k[i];
        if (stage == 3) {
            U[i] += dt * (acc[i] + b[3] * kv);
        } else {
            const double a = (stage == 0 ? 0.0 : acc[i]) + b[stage] * kv;
            acc[i] = a;
            us[i] = U[i] + cnext[stage] * dt * kv;
        }
    }
}

// Reduced precisions. GB300 runs FP64 arithmetic and FP32<->FP64 conversions on its FP64 pipe, at
// 1/64 of the FP32 rate, so the stage updates keep FP64 work to the two places that need it: at
// the start of a step the FP64 master state U is rounded once to FP32, hi = fl32(U); stage states
// u_{s+1} = hi + c_{s+1} dt k_s and the Runge-Kutta sum acc = sum b_s k_s are formed in FP32; the
// last stage adds the increment dt (acc + b_3 k_3) to U in FP64. A stage state thus differs from
// fl32(U + c dt k) by at most about one FP32 rounding (it is an FP32 input of the RHS either way);
// the increments carry an FP32 rounding on top of that of k itself; U stays FP64.
template <typename T>
__global__ void k_rk_split(const double *__restrict__ U, float *__restrict__ hi, T *__restrict__ us, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float h = (float)U[i];
        hi[i] = h;
        us[i] = (T)h;
    }
}

// After stage s (k = R(u_s)): acc (+)= b_s k; u_{s+1} = hi + c_{s+1} dt k; the last stage updates U.
template <typename T>
__global__ void k_rk_update(double *__restrict__ U, const T *__restrict__ k, float *__restrict__ acc, const float *__restrict__ hi,
                            T *__restrict__ us, long long n, double dt, float cdt, float b, int stage)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float kv = (float)k[i];
        if (stage == 3) {
            U[i] += dt * (double)(acc[i] + b * kv);
        } else {
            acc[i] = (stage == 0 ? 0.0f : acc[i]) + b * kv;
            us[i] = (T)(hi[i] + cdt * kv);
        }
    }
}

// The same steps with the stage arithmetic in FP64 (fr_set_rk_fp64_stages): the stage states
// u_{s+1} = fl(U + c_{s+1} dt k_s) and the sum acc = sum b_s k_s are formed in FP64 from the FP64
// master state, as in the FP64 form; only the RHS evaluations run in the reduced precision. At the
// start of a step the RHS input is fl(U).
template <typename T>
__global__ void k_rk_cast(const double *__restrict__ U, T *__restrict__ us, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        us[i] = (T)U[i];
}

template <typename T>
__global__ void k_rk_update_wide(double *__restrict__ U, const T *__restrict__ k, double *__restrict__ acc,
                                 T *__restrict__ us, long long n, double dt, int stage)
{
    const double b[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    const double cnext[4] = {0.5, 0.5, 1.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const double kv = (double)k[i];
        if (stage == 3) {
            U[i] += dt * (acc[i] + b[3] * kv);
        } else {
            acc[i] = (stage == 0 ? 0.0 : acc[i]) + b[stage] * kv;
            us[i] = (T)(U[i] + cnext[stage] * dt * kv);
        }
    }
}

// One RK4 stage st (0..3) of the step U -> U + dt sum_s b_s k_s, or one phase of it (only = 0, 1, 2:
// face solution, volume group, interface group with the stage update; only < 0: all of it). The
// stage's RHS input is U (FP64) or fl32(U) (reduced precisions, split off at the start of stage 0)
// for st = 0 and the stage state us otherwise.
template <typename T>
static fr_status rk4_enqueue_stage(fr_mesh *m, double *U, double dt, cudaStream_t s, int st, int only)
{
    const long long n = m->nU;
    const int thr = 256;
    const int grid = (int)std::min<long long>((n + thr - 1) / thr, 16LL * m->nsm);
    // reduced precisions: d_rk_acc holds the FP32 Runge-Kutta sum and fl32(U)
    float *accf = reinterpret_cast<float *>(m->d_rk_acc);
    float *uhi = m->prec == FR_FP64 ? nullptr : accf + n;
    const void *u0 = U;
    if (m->prec != FR_FP64) {
        if (st == 0 && only <= 0) {
            if (m->rk_wide) k_rk_cast<T><<<grid, thr, 0, s>>>(U, reinterpret_cast<T *>(m->d_rk_us), n);
            else k_rk_split<T><<<grid, thr, 0, s>>>(U, uhi, reinterpret_cast<T *>(m->d_rk_us), n);
        }
        u0 = m->d_rk_us;
    }
    const void *in = st == 0 ? u0 : m->d_rk_us;
    if (m->form == FR_FUSED && m->prec == FR_FP64) {
        // FP64: the stage update is folded into the interface kernel (no RHS array, no extra
        // launch). The reduced precisions write R and run the update as its own streaming
        // kernel: their latency-bound interface kernels would stall on the FP64 master-state
        // and accumulator traffic, which the element-wise kernel moves near the HBM peak.
        RkFold rk;
        rk.stage = st; rk.dt = dt; rk.U = U; rk.acc = m->d_rk_acc; rk.us = m->d_rk_us;
        fr_status r = rhs_impl<T>(m, in, m->d_rk_k, s, rk, only);
        if (r) return r;
        CU(cudaPeekAtLastError());
        return FR_OK;
    }
    fr_status r = only < 0 ? rhs_dispatch(m, in, m->d_rk_k, s) : rhs_impl<T>(m, in, m->d_rk_k, s, RkFold(), only);
    if (r) return r;
    if (only >= 0 && only != 2) return FR_OK;
    TimeScope ts(m, 30, s);
    if constexpr (sizeof(T) == 8) {
        k_rk_update64<<<grid, thr, 0, s>>>(U, reinterpret_cast<const double *>(m->d_rk_k), m->d_rk_acc,
                                           reinterpret_cast<double *>(m->d_rk_us), n, dt, st);
    } else if (m->rk_wide) {
        k_rk_update_wide<T><<<grid, thr, 0, s>>>(U, reinterpret_cast<const T *>(m->d_rk_k), m->d_rk_acc,
                                                 reinterpret_cast<T *>(m->d_rk_us), n, dt, st);
    } else {
        const double bs[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0}, cnext[4] = {0.5, 0.5, 1.0, 0.0};
        k_rk_update<T><<<grid, thr, 0, s>>>(U, reinterpret_cast<const T *>(m->d_rk_k), accf, uhi,
                                            reinterpret_cast<T *>(m->d_rk_us), n, dt, (float)(cnext[st] * dt),
                                            (float)bs[st], st);
    }
    CU(cudaPeekAtLastError());
    return FR_OK;
}

template <typename T>
static fr_status rk4_enqueue_step(fr_mesh *m, double *U, double dt, cudaStream_t s)
{
    for (int st = 0; st < 4; st++) {
        fr_status r = rk4_enqueue_stage<T>(m, U, dt, s, st, -1);
        if (r) return r;
    }
    return FR_OK;
}

template <typename T>
static fr_status rk4_impl(fr_mesh *m, double *U, double dt, int nsteps, cudaStream_t s)
{
    // Graph replay needs a capturable stream: the legacy default stream (NULL) is not, and per-kernel
    // timing records host-visible events, so both run the launches directly.
    if (!m->use_graph || m->timing || s == nullptr) {
        for (int step = 0; step < nsteps; step++) {
            fr_status r = rk4_enqueue_step<T>(m, U, dt, s);
            if (r) return r;
        }
        return FR_OK;
    }
    int done = 0;
    const int gform = m->form + 2 * m->hex_tc + 4 * m->dense_tc;
    if (!m->graph || m->graph_U != U || m->graph_dt != dt || m->graph_stream != s || m->graph_form != gform) {
        if (m->graph) { cudaGraphExecDestroy(m->graph); m->graph = nullptr; }
        // one eager step first: lazy workspace allocation and first-launch kernel attributes happen
        // outside the capture
        fr_status r0 = rk4_enqueue_step<T>(m, U, dt, s);
        if (r0) return r0;
        done = 1;
        if (nsteps <= 1) return FR_OK;
        cudaGraph_t g = nullptr;
        CU(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        fr_status r = rk4_enqueue_step<T>(m, U, dt, s);
        cudaError_t ce = cudaStreamEndCapture(s, &g);
        if (r) { if (g) cudaGraphDestroy(g); return r; }
        if (ce != cudaSuccess) return fail(FR_ECUDA, "RK4 graph capture: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&m->graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) { m->graph = nullptr; return fail(FR_ECUDA, "RK4 graph instantiate: %s", cudaGetErrorString(ce)); }
        m->graph_U = U; m->graph_dt = dt; m->graph_stream = s; m->graph_form = gform;
    }
    for (int step = done; step < nsteps; step++) CU(cudaGraphLaunch(m->graph, s));
    return FR_OK;
}

static fr_status rk4_buffers(fr_mesh *m)
{
    size_t ts = tsize(m->prec);
    fr_status st = dalloc(m, &m->d_rk_k, (size_t)m->nU * ts);
    if (!st) st = dalloc(m, &m->d_rk_us, (size_t)m->nU * ts);
    // FP64 (and reduced precisions with FP64 stage arithmetic): the Runge-Kutta sum; reduced
    // precisions otherwise: its FP32 form and fl32(U) (the same bytes)
    if (!st) st = dalloc(m, (void **)&m->d_rk_acc, (size_t)m->nU * sizeof(double));
    return st;
}

extern "C" fr_status fr_rk4_stage(fr_mesh *m, int stage, int phase, void *U_dev, double dt, void *stream)
{
    if (!m || !U_dev || stage < 0 || stage > 3 || phase < 0 || phase > 2 || !(dt == dt))
        return fail(FR_EINVAL, "bad argument");
    if (m->form != FR_FUSED) return fail(FR_EUNSUPPORTED, "fr_rk4_stage runs the fused form");
    fr_status st = check_status(m);
    if (!st) st = rk4_buffers(m);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = m->prec == FR_FP64 ? rk4_enqueue_stage<double>(m, (double *)U_dev, dt, s, stage, phase)
                            : rk4_enqueue_stage<float>(m, (double *)U_dev, dt, s, stage, phase);
    if (st) return st;
    return phase == 2 ? post_status(m, s) : FR_OK;
}

extern "C" fr_status fr_rk4_step(fr_mesh *m, void *U_dev, double dt, int nsteps, void *stream)
{
    if (!m || !U_dev || nsteps < 0 || !(dt == dt)) return fail(FR_EINVAL, "bad argument");
    if (m->nparts > 1)
        return fail(FR_EUNSUPPORTED, "a partitioned mesh advances through fr_rk4_stage and halo exchanges");
    fr_status st = check_status(m);
    if (st) return st;
    st = rk4_buffers(m);
    if (st) return st;
    cudaStream_t s = (cudaStream_t)stream;
    st = m->prec == FR_FP64 ? rk4_impl<double>(m, (double *)U_dev, dt, nsteps, s) : rk4_impl<float>(m, (double *)U_dev, dt, nsteps, s);
    if (st) return st;
    return post_status(m, s);
}

extern "C" fr_status fr_rk4_step_host(fr_mesh *m, void *U_host, double dt, int nsteps, void *stream)
{
    if (!m || !U_host) return fail(FR_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = (size_t)m->nU * sizeof(double);
    fr_status st = dalloc(m, &m->d_io_U, std::max(bytes, (size_t)m->nU * tsize(m->prec)));
    if (st) return st;
    CU(cudaMemcpyAsync(m->d_io_U, U_host, bytes, cudaMemcpyHostToDevice, s));
    st = fr_rk4_step(m, m->d_io_U, dt, nsteps, stream);
    if (st) return st;
    CU(cudaMemcpyAsync(U_host, m->d_io_U, bytes, cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    return check_status(m);
}

// ---------------------------------------------------------------------------------------------
// Info, coordinates, diagnostics, stages
// ---------------------------------------------------------------------------------------------
extern "C" long long fr_num_values(const fr_mesh *m) { return m ? m->nU : 0; }

extern "C" fr_status fr_mesh_info(const fr_mesh *m, long long *info)
{
    if (!m || !info) return fail(FR_EINVAL, "null argument");
    info[0] = m->ne; info[1] = m->nU; info[2] = m->nfpt; info[3] = m->npair; info[4] = (long long)m->inst.size();
    info[5] = m->form != FR_FUSED ? 13 : (m->merged && can_merge(m)) ? 3 : (m->split_c ? 4 : 3) * (long long)m->groups.size();
    info[6] = m->bytes;
    return FR_OK;
}

extern "C" fr_status fr_instance_offsets(const fr_mesh *m, long long *off)
{
    if (!m || !off) return fail(FR_EINVAL, "null argument");
    for (size_t i = 0; i < m->inst_u0.size(); i++) off[i] = m->inst_u0[i];
    return FR_OK;
}

extern "C" fr_status fr_sol_coords(const fr_mesh *m, double *xyz)
{
    if (!m || !xyz) return fail(FR_EINVAL, "null argument");
    long long k = 0;
    for (size_t b = 0; b < m->blocks.size(); b++) {
        const Block &B = m->blocks[b];
        const InstanceHost &I = m->inst[B.inst];
        const frb::Hex1D &h = m->hex1d[b];
        int n = h.n;
        long long le0 = B.type == 0 ? 0 : (B.type == 1 ? I.n_hex : (B.type == 2 ? I.n_hex + I.n_pri : I.n_hex + I.n_pri + I.n_tet));
        for (long long e = 0; e < B.ne; e++) {
            for (int z = 0; z < B.nu; z++, k++) {
                double X[3];
                if (B.type == 0) { X[0] = h.x[z % n]; X[1] = h.x[(z / n) % n]; X[2] = h.x[z / (n * n)]; }
                else if (B.type == 1) { X[0] = m->pri.xt[z % FR_PT][0]; X[1] = m->pri.xt[z % FR_PT][1]; X[2] = h.x[z / FR_PT]; }
                else if (B.type == 2) { X[0] = m->tet.x[z][0]; X[1] = m->tet.x[z][1]; X[2] = m->tet.x[z][2]; }
                else { X[0] = m->pyr.x[z][0]; X[1] = m->pyr.x[z][1]; X[2] = m->pyr.x[z][2]; }
                map_point(I, le0 + e, X, xyz + 3 * k);
            }
        }
    }
    return FR_OK;
}

struct WPts {
    double w[FR_MAXN * FR_MAXN * FR_MAXN];   // quadrature weight of every solution point
};

// Per-element partial sums of the diagnostics; out[k] (k < 8): 0 volume, 1 int rho|v|^2/2,
// 2 -int d(rho|v|^2/2)/dt from R, 3..7 int R_alpha (weights W = tensor GL weights times detJ).
template <typename T>
__global__ void k_diag(const T *__restrict__ U, const T *__restrict__ R, const Geo<T> *__restrict__ geo, long long ne,
                       int NU, WPts wp, double *out, const T *__restrict__ mu)
{
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long e = blockIdx.x; e < ne; e += gridDim.x) {
        const T *u = U + e * 5 * NU;
        const T *r = R ? R + e * 5 * NU : nullptr;
        const double det = (double)geo[e].det;
        for (int z = threadIdx.x; z < NU; z += blockDim.x) {
            // curved elements: det J at the solution point
            const double w = wp.w[z] * (mu ? (double)mu[(e * NU + z) * 10 + 9] : det);
            const double rho = (double)u[z];
            const double v0 = (double)u[NU + z] / rho, v1 = (double)u[2 * NU + z] / rho, v2 = (double)u[3 * NU + z] / rho;
            const double v2s = v0 * v0 + v1 * v1 + v2 * v2;
            acc[0] += w;
            acc[1] += w * 0.5 * rho * v2s;
            if (r) {
                acc[2] -= w * (v0 * (double)r[NU + z] + v1 * (double)r[2 * NU + z] + v2 * (double)r[3 * NU + z] - 0.5 * v2s * (double)r[z]);
                for (int a = 0; a < 5; a++) acc[3 + a] += w * (double)r[a * NU + z];
            }
        }
    }
    for (int k = 0; k < 8; k++) {
        double v = acc[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(&out[k], v);
    }
}

extern "C" fr_status fr_diagnostics(fr_mesh *m, const void *U, const void *R, double *out, void *stream)
{
    if (!m || !U || !out) return fail(FR_EINVAL, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    size_t ni = m->inst.size();
    fr_status st = dalloc(m, (void **)&m->d_wsum, ni * 8 * sizeof(double));
    if (st) return st;
    CU(cudaMemsetAsync(m->d_wsum, 0, ni * 8 * sizeof(double), s));
    for (size_t bi = 0; bi < m->blocks.size(); bi++) {
        const Block &b = m->blocks[bi];
        WPts wp{};
        const frb::Hex1D &h = m->hex1d[bi];
        for (int z = 0; z < b.nu; z++)
            wp.w[z] = b.type == 0 ? h.w[z % h.n] * h.w[(z / h.n) % h.n] * h.w[z / (h.n * h.n)]
                    : b.type == 1 ? m->pri.wt[z % FR_PT] * h.w[z / FR_PT] : (b.type == 2 ? m->tet.w[z] : m->pyr.w[z]);
        int grid = (int)std::min<long long>(std::max<long long>(b.ne, 1), 8LL * m->nsm);
        double *o = m->d_wsum + 8 * b.inst;
        size_t ts = tsize(m->prec);
        const char *u = (const char *)U + b.u0 * ts;
        const char *r = R ? (const char *)R + b.u0 * ts : nullptr;
        if (m->prec == FR_FP64)
            k_diag<double><<<grid, 128, 0, s>>>((const double *)u, (const double *)r,
                                                 (const Geo<double> *)m->d_geo + b.elem0, b.ne, b.nu, wp, o,
                                                 (const double *)m->d_mu);
        else
            k_diag<float><<<grid, 128, 0, s>>>((const float *)u, (const float *)r,
                                                (const Geo<float> *)m->d_geo + b.elem0, b.ne, b.nu, wp, o,
                                                (const float *)m->d_mu);
        CU(cudaPeekAtLastError());
    }
    std::vector<double> h(ni * 8);
    CU(cudaMemcpyAsync(h.data(), m->d_wsum, ni * 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (size_t i = 0; i < ni; i++) {
        const double *a = &h[8 * i];
        double *o = out + 8 * i;
        o[0] = a[0];
        o[1] = a[0] > 0 ? a[1] / a[0] : 0.0;   // an instance without elements has no mean
        o[2] = a[0] > 0 ? a[2] / a[0] : 0.0;
        for (int k = 0; k < 5; k++) o[3 + k] = a[3 + k];
    }
    return FR_OK;
}

// ---------------------------------------------------------------------------------------------
// Diagnostics without any allocation
//
// fr_diagnostics allocates its device accumulators with cudaMalloc on first use. Callers that must
// not allocate device memory -- code running while another framework owns the device memory budget,
// a real-time loop that cannot afford the device-wide synchronisation a cudaMalloc may cause, or a
// thread that is capturing other work into a CUDA graph in global capture mode, where cudaMalloc is
// not allowed -- use fr_diagnostics_noalloc instead. Its accumulators live in the fixed array below,
// which every GPU that loads this library holds until the process exits.
// ---------------------------------------------------------------------------------------------
#define FR_NOALLOC_MAX_INST 1024
static __device__ __align__(256) double g_diag_scratch[FR_NOALLOC_MAX_INST * 8];

// Device address of g_diag_scratch per device (the host-side symbol is only a stand-in and must
// never be handed to a kernel). fr_mesh_create looks it up with the handle's device current, so every
// live handle finds the address of the current context's copy, also after a cudaDeviceReset.
static double *g_diag_ptrs[64] = {nullptr};

static cudaError_t diag_scratch_lookup(int dev)
{
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    double *p = nullptr;
    const cudaError_t err = cudaGetSymbolAddress((void **)&p, g_diag_scratch);
    g_diag_ptrs[dev] = err == cudaSuccess ? p : nullptr;
    return err;
}

extern "C" fr_status fr_diagnostics_noalloc(fr_mesh *m, const void *U, const void *R, double *out, void *stream)
{
    if (!m || !U || !out) return fail(FR_EINVAL, "null argument");
    const int ni = (int)m->inst.size();
    if (ni > FR_NOALLOC_MAX_INST)
        return fail(FR_EINVAL, "fr_diagnostics_noalloc: %d instances exceed the fixed scratch limit of %d", ni,
                    FR_NOALLOC_MAX_INST);
    int dev = 0;
    CU(cudaGetDevice(&dev));
    if (dev != m->dev)
        return fail(FR_EINVAL, "fr_diagnostics_noalloc: device %d is current, the handle lives on device %d", dev, m->dev);
    double *acc = g_diag_ptrs[dev];
    if (!acc) return fail(FR_ECUDA, "fr_diagnostics_noalloc: no device address of the diagnostics array");
    cudaStream_t s = (cudaStream_t)stream;
    // the array keeps the previous call's sums: clear the slots this call accumulates into
    CU(cudaMemsetAsync(acc, 0, (size_t)ni * 8 * sizeof(double), s));
    for (size_t bi = 0; bi < m->blocks.size(); bi++) {
        const Block &b = m->blocks[bi];
        WPts wp{};
        const frb::Hex1D &h = m->hex1d[bi];
        for (int z = 0; z < b.nu; z++)
            wp.w[z] = b.type == 0 ? h.w[z % h.n] * h.w[(z / h.n) % h.n] * h.w[z / (h.n * h.n)]
                    : b.type == 1 ? m->pri.wt[z % FR_PT] * h.w[z / FR_PT] : (b.type == 2 ? m->tet.w[z] : m->pyr.w[z]);
        int grid = (int)std::min<long long>(std::max<long long>(b.ne, 1), 8LL * m->nsm);
        double *o = acc + 8 * b.inst;
        size_t ts = tsize(m->prec);
        const char *u = (const char *)U + b.u0 * ts;
        const char *r = R ? (const char *)R + b.u0 * ts : nullptr;
        if (m->prec == FR_FP64)
            k_diag<double><<<grid, 128, 0, s>>>((const double *)u, (const double *)r,
                                                 (const Geo<double> *)m->d_geo + b.elem0, b.ne, b.nu, wp, o,
                                                 (const double *)m->d_mu);
        else
            k_diag<float><<<grid, 128, 0, s>>>((const float *)u, (const float *)r,
                                                (const Geo<float> *)m->d_geo + b.elem0, b.ne, b.nu, wp, o,
                                                (const float *)m->d_mu);
        CU(cudaPeekAtLastError());
    }
    // raw sums straight into the caller's array, then normalised in place (no host buffer either)
    CU(cudaMemcpyAsync(out, acc, (size_t)ni * 8 * sizeof(double), cudaMemcpyDeviceToHost, s));
    CU(cudaStreamSynchronize(s));
    for (int i = 0; i < ni; i++) {
        double *o = out + 8 * i;
        o[1] = o[0] > 0 ? o[1] / o[0] : 0.0;   // an instance without elements has no mean
        o[2] = o[0] > 0 ? o[2] / o[0] : 0.0;
    }
    return FR_OK;
}

extern "C" fr_status fr_stage(fr_mesh *m, int which, double *host, long long n_host, long long *n_needed)
{
    if (!m) return fail(FR_EINVAL, "null handle");
    void *src = nullptr;
    long long n = 0;
    const Block &b = m->blocks[0];
    switch (which) {
    case 0: src = m->d_UF; n = 5 * m->nfpt; break;
    case 1: src = m->d_CF; n = 5 * m->nfpt; break;
    case 2: src = m->d_Qsnap; n = 15 * b.ne * b.nu; break;
    case 3: src = m->d_QF; n = 15 * m->nfpt; break;
    case 4: src = m->d_Qu; n = 15 * b.ne * b.nu; break;
    case 5: src = m->d_DF; n = 5 * m->nfpt; break;
    default: return fail(FR_EINVAL, "unknown stage %d", which);
    }
    if (n_needed) *n_needed = n;
    if (!host) return FR_OK;
    if (!src) return fail(FR_EINVAL, "stage %d has not been computed (run an unfused RHS first)", which);
    if (n_host < n) return fail(FR_EINVAL, "host buffer too small");
    CU(cudaDeviceSynchronize());
    if (m->prec == FR_FP64) {
        CU(cudaMemcpy(host, src, n * sizeof(double), cudaMemcpyDeviceToHost));
    } else {
        std::vector<float> tmp((size_t)n);
        CU(cudaMemcpy(tmp.data(), src, n * sizeof(float), cudaMemcpyDeviceToHost));
        for (long long i = 0; i < n; i++) host[i] = tmp[i];
    }
    return FR_OK;
}
