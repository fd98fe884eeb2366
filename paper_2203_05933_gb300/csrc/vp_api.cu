// C ABI of libvp (declared in include/vp.h): plan construction, evaluation,
// adjoint, inspection. Host code only; kernels live in vp_fmm.cu (Laplace FMM),
// vp_mhelm.cu (modified-Helmholtz FMM), vp_spmv.cu (correction apply),
// vp_upsample.cu, vp_interp.cu, vp_tricorr.cu and vp_static.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "vp_internal.h"

using namespace vp;

namespace {

thread_local std::string g_last_error;

vp_status fail(vp_status st, const std::string& msg)
{
    g_last_error = msg;
    return st;
}

vp_status cuda_fail(cudaError_t e, const char* where)
{
    g_last_error = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? VP_ERR_OOM : VP_ERR_CUDA;
}

#define VP_CUDA(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

uint64_t binom_u64(int n, int k)
{
    if (k < 0 || k > n) return 0;
    uint64_t r = 1;
    for (int i = 1; i <= k; ++i) r = r * (uint64_t)(n - k + i) / (uint64_t)i;  // exact at every step
    return r;
}

// Operator tables for order P, laid out as in DevTables (all offsets multiples of 2 doubles).
std::vector<double> make_tables(int P, size_t off[7])
{
    const int P1 = P + 1;
    std::vector<double> v;
    auto reserve_even = [&]() {
        if (v.size() & 1) v.push_back(0.0);
    };
    off[0] = v.size();  // H
    for (int l = 0; l <= P; ++l)
        for (int k = 0; k <= P; ++k) v.push_back(k >= 1 ? (double)binom_u64(l + k - 1, k - 1) : 0.0);
    off[1] = v.size();  // Bm
    for (int l = 0; l <= P; ++l)
        for (int k = 0; k <= P; ++k)
            v.push_back((k >= 1 && k <= l) ? std::ldexp((double)binom_u64(l - 1, k - 1), -k) : 0.0);
    off[2] = v.size();  // Bl
    for (int l = 0; l <= P; ++l)
        for (int k = 0; k <= P; ++k) v.push_back(k >= l ? std::ldexp((double)binom_u64(k, l), -l) : 0.0);
    reserve_even();
    off[3] = v.size();  // tpow [49][P1] complex
    std::vector<double> mt;
    for (int oy = -3; oy <= 3; ++oy)
        for (int ox = -3; ox <= 3; ++ox) {
            const bool far = std::max(std::abs(ox), std::abs(oy)) >= 2;
            const long double den = 2.0L * (long double)(ox * ox + oy * oy);
            const long double tr = far ? (long double)ox / den : 0.0L;
            const long double ti = far ? -(long double)oy / den : 0.0L;
            long double pr = 1.0L, pi = 0.0L;  // t^l
            long double mr = 1.0L, mi = 0.0L;  // (-t)^l
            for (int l = 0; l <= P; ++l) {
                v.push_back(far ? (double)pr : 0.0);
                v.push_back(far ? (double)pi : 0.0);
                mt.push_back(far ? (double)mr : 0.0);
                mt.push_back(far ? (double)mi : 0.0);
                const long double nr = pr * tr - pi * ti, ni = pr * ti + pi * tr;
                pr = nr;
                pi = ni;
                const long double qr = -(mr * tr - mi * ti), qi = -(mr * ti + mi * tr);
                mr = qr;
                mi = qi;
            }
        }
    off[4] = v.size();  // mtpow
    v.insert(v.end(), mt.begin(), mt.end());
    off[5] = v.size();  // log2o [49]
    for (int oy = -3; oy <= 3; ++oy)
        for (int ox = -3; ox <= 3; ++ox) {
            const int r2 = ox * ox + oy * oy;
            v.push_back(r2 > 0 ? std::log(2.0) + 0.5 * std::log((double)r2) : 0.0);
        }
    reserve_even();
    off[6] = v.size();  // zpow [4][P1] complex
    for (int c = 0; c < 4; ++c) {
        const double zr = (c & 1) ? 0.5 : -0.5, zi = (c & 2) ? 0.5 : -0.5;
        double pr = 1.0, pi = 0.0;
        for (int m = 0; m <= P; ++m) {
            v.push_back(pr);
            v.push_back(pi);
            const double nr = pr * zr - pi * zi, ni = pr * zi + pi * zr;  // exact: dyadic values
            pr = nr;
            pi = ni;
        }
    }
    (void)P1;
    return v;
}

// 128-entry table for the float-float log of the near-field kernel: for
// c_k = 1 + (k + 1/2)/128, rc_k = fl(1/c_k) and T_k = -log(rc_k) split as
// T_hi (rounded to 19 fractional bits, so that e*ln2_hi + T_hi is exact in one
// float for |e| <= 15) plus T_lo.
std::vector<float> make_log_table()
{
    std::vector<float> t(128 * 4);
    for (int k = 0; k < 128; ++k) {
        const long double c = 1.0L + ((long double)k + 0.5L) / 128.0L;
        const float rc = (float)(1.0L / c);
        const long double T = -logl((long double)rc);
        const long double Th = roundl(T * 524288.0L) / 524288.0L;
        t[4 * k + 0] = rc;
        t[4 * k + 1] = (float)Th;
        t[4 * k + 2] = (float)(T - Th);
        t[4 * k + 3] = 0.0f;
    }
    return t;
}

// Float-float copies of the M2L tables (each value split as hi + lo floats):
// H [P1][P1] (float2), t^l and (-t)^k [49][P1] (float4 complex), log(2|o|) [49],
// 1/l [P1] (float2), the M2M and L2L binomials [P1][P1] (float2) and the child
// offset powers zeta^m [4][P1] (float2, exact). Offsets in floats in off[8].
std::vector<float> make_ff_tables(int P, size_t off[8])
{
    const int P1 = P + 1;
    std::vector<float> v;
    auto split = [&](long double x) {
        const float h = (float)x;
        v.push_back(h);
        v.push_back((float)(x - (long double)h));
    };
    auto align16 = [&]() {  // every table starts on a 16-byte boundary (float4 loads)
        while (v.size() % 4) v.push_back(0.0f);
    };
    off[0] = v.size();
    for (int l = 0; l <= P; ++l)
        for (int k = 0; k <= P; ++k) {
            if (k == 0) {
                split(0.0L);
                continue;
            }
            const uint64_t hb = binom_u64(l + k - 1, k - 1);
            const float h = (float)hb;
            v.push_back(h);
            v.push_back((float)((long double)hb - (long double)h));
        }
    for (int pass = 0; pass < 2; ++pass) {
        align16();
        off[1 + pass] = v.size();
        for (int oy = -3; oy <= 3; ++oy)
            for (int ox = -3; ox <= 3; ++ox) {
                const bool far = std::max(std::abs(ox), std::abs(oy)) >= 2;
                const long double den = 2.0L * (long double)(ox * ox + oy * oy);
                const long double sgn = pass == 0 ? 1.0L : -1.0L;
                const long double tr = far ? sgn * (long double)ox / den : 0.0L;
                const long double ti = far ? -sgn * (long double)oy / den : 0.0L;
                long double pr = 1.0L, pi = 0.0L;
                for (int l = 0; l <= P; ++l) {
                    split(far ? pr : 0.0L);
                    split(far ? pi : 0.0L);
                    const long double nr = pr * tr - pi * ti, ni = pr * ti + pi * tr;
                    pr = nr;
                    pi = ni;
                }
            }
    }
    align16();
    off[3] = v.size();
    for (int oy = -3; oy <= 3; ++oy)
        for (int ox = -3; ox <= 3; ++ox) {
            const int r2 = ox * ox + oy * oy;
            split(r2 > 0 ? logl(2.0L) + 0.5L * logl((long double)r2) : 0.0L);
        }
    align16();
    off[4] = v.size();
    for (int l = 0; l <= P; ++l) split(l == 0 ? 0.0L : 1.0L / (long double)l);
    align16();
    off[5] = v.size();
    for (int l = 0; l <= P; ++l)
        for (int k = 0; k <= P; ++k)
            split((k >= 1 && k <= l) ? ldexpl((long double)binom_u64(l - 1, k - 1), -k) : 0.0L);
    align16();
    off[6] = v.size();
    for (int l = 0; l <= P; ++l)
        for (int k = 0; k <= P; ++k) split(k >= l ? ldexpl((long double)binom_u64(k, l), -l) : 0.0L);
    align16();
    off[7] = v.size();
    for (int c = 0; c < 4; ++c) {
        const double zr = (c & 1) ? 0.5 : -0.5, zi = (c & 2) ? 0.5 : -0.5;
        double pr = 1.0, pi = 0.0;
        for (int m = 0; m <= P; ++m) {
            v.push_back((float)pr);  // exact: dyadic values
            v.push_back((float)pi);
            const double nr = pr * zr - pi * zi, ni = pr * zi + pi * zr;
            pr = nr;
            pi = ni;
        }
    }
    (void)P1;
    return v;
}

// For each entry (b, A) of an interaction list: the centre of box A relative to
// the centre of box b in units of b's side, and side_A / side_b. Both are exact
// dyadic numbers: with dl = level_b - level_A,
// (c_A - c_b)/side_b = K 2^(min(dl,0) - 1), K = (2 ix_A + 1) 2^max(dl,0) - (2 ix_b + 1) 2^max(-dl,0).
std::vector<float> make_list_offsets(const Tree& T, const std::vector<int32_t>& ptr, const std::vector<int32_t>& idx)
{
    std::vector<float> o(idx.size() * 4, 0.0f);
    for (int64_t b = 0; b + 1 < (int64_t)ptr.size(); ++b)
        for (int32_t e = ptr[(size_t)b]; e < ptr[(size_t)b + 1]; ++e) {
            const int32_t a = idx[(size_t)e];
            const int dl = T.level[(size_t)b] - T.level[(size_t)a];
            const int up = dl > 0 ? dl : 0, dn = dl < 0 ? -dl : 0;
            const int64_t kx = (2LL * T.ix[(size_t)a] + 1) * (1LL << up) - (2LL * T.ix[(size_t)b] + 1) * (1LL << dn);
            const int64_t ky = (2LL * T.iy[(size_t)a] + 1) * (1LL << up) - (2LL * T.iy[(size_t)b] + 1) * (1LL << dn);
            o[4 * (size_t)e + 0] = (float)std::ldexp((double)kx, (dl < 0 ? dl : 0) - 1);
            o[4 * (size_t)e + 1] = (float)std::ldexp((double)ky, (dl < 0 ? dl : 0) - 1);
            o[4 * (size_t)e + 2] = (float)std::ldexp(1.0, dl);
        }
    return o;
}

// Leaf-relative coordinates of every point of each leaf: ((x, y) - centre)/side,
// each component split into hi + lo floats, hi on the grid 2^-21.
std::vector<float> make_rho(const Tree& T, const std::vector<double>& xy_sorted, bool sources)
{
    const size_t n = xy_sorted.size() / 2;
    std::vector<float> r(n * 4, 0.0f);
    for (int64_t b = 0; b < T.n_boxes(); ++b) {
        if (!T.is_leaf[(size_t)b]) continue;
        const int32_t p0 = sources ? T.src_begin[(size_t)b] : T.tgt_begin[(size_t)b];
        const int32_t p1 = sources ? T.src_end[(size_t)b] : T.tgt_end[(size_t)b];
        const double side = T.box_side((int)b), cx = T.box_cx((int)b), cy = T.box_cy((int)b);
        for (int32_t i = p0; i < p1; ++i) {
            const double rx = (xy_sorted[2 * (size_t)i] - cx) / side;
            const double ry = (xy_sorted[2 * (size_t)i + 1] - cy) / side;
            // hi parts on the grid 2^-21: |rho| <= 1/2 needs 20 bits, and after the
            // exact shift/scale to a neighbouring leaf one level apart (factor 1/2
            // or 2) the difference of two hi parts still fits 24 bits
            const float xh = (float)(std::nearbyint(rx * 2097152.0) / 2097152.0);
            const float yh = (float)(std::nearbyint(ry * 2097152.0) / 2097152.0);
            r[4 * (size_t)i + 0] = xh;
            r[4 * (size_t)i + 1] = (float)(rx - (double)xh);
            r[4 * (size_t)i + 2] = yh;
            r[4 * (size_t)i + 3] = (float)(ry - (double)yh);
        }
    }
    return r;
}

bool finite_all(const std::vector<double>& a)
{
    for (double x : a)
        if (!std::isfinite(x)) return false;
    return true;
}

}  // namespace

namespace vp {
void set_last_error(const std::string& msg) { g_last_error = msg; }
std::vector<float> log_table() { return make_log_table(); }
}  // namespace vp

// ---------------------------------------------------------------------------
int PhaseTimer::begin(const char* name)
{
    if (!on) return -1;
    int ph = -1;
    for (size_t i = 0; i < names.size(); ++i)
        if (names[i] == name) ph = (int)i;
    if (ph < 0) {
        names.emplace_back(name);
        ph = (int)names.size() - 1;
    }
    if ((size_t)(2 * used + 2) > pool.size()) {
        for (int k = 0; k < 16; ++k) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return -1;
            pool.push_back(e);
        }
    }
    const int id = used++;
    if ((size_t)id >= phase_of.size()) phase_of.resize(id + 1);
    phase_of[id] = ph;
    cudaEventRecord(pool[2 * id], stream);
    return id;
}

void PhaseTimer::end(int id)
{
    if (id < 0) return;
    cudaEventRecord(pool[2 * id + 1], stream);
}

struct vp_plan_s {
    int device = 0;
    int P = 30;
    int leaf = 64;
    int max_dens = 1;
    int nd_cap = 1;
    uint32_t flags = 0;
    Arith arith = Arith::kF64;  // fixed at creation from VP_FLAG_FF / VP_FLAG_FP64
    int64_t n_src = 0, n_tgt = 0, nnz = 0;
    int64_t n_f = 0;            // density length: n_src, or the p-nodes of an upsampled plan
    bool ups = false;           // charges interpolated per cell from the p-nodes (oversampling)
    DevUpsample dups;
    int32_t n_problems = 1;
    int32_t stat_levels = 0;
    int64_t stat_boxes = 0, stat_leaves = 0, stat_u = 0, stat_v = 0, stat_w = 0, stat_x = 0;
    double stat_root[3] = {0.0, 0.0, 0.0};
    DevTree dt;
    DevTables tab;
    std::vector<void*> allocs;
    // points and weights in tree order
    double2* src_xy = nullptr;
    double2* tgt_xy = nullptr;
    longlong2* src_fix = nullptr;  // the same points on the integer grid 2^-fix_sigma
    longlong2* tgt_fix = nullptr;
    int fix_sigma = 60;
    double2* src_pow = nullptr;    // powers of the points relative to their leaves, [n][P] (float64 plans)
    double2* tgt_pow = nullptr;
    float4* src_rho = nullptr;
    float4* tgt_rho = nullptr;
    double* w_sorted = nullptr;
    int32_t *src_perm = nullptr, *tgt_perm = nullptr, *src_inv = nullptr, *tgt_inv = nullptr;
    int32_t *box_src = nullptr, *box_tgt = nullptr;
    // correction in caller order, and its transpose
    int64_t* rowptr = nullptr;
    int32_t* col = nullptr;
    double* val = nullptr;
    int64_t* cptr = nullptr;
    int32_t* crow = nullptr;
    double* cval = nullptr;
    bool grouped = false;       // correction applied by a grouped kernel (float64, or float-float with VP_FLAG_FF)
    DevGroupedCSR gfwd;         // Pi, rows grouped by shared column lists (Pi^T g from the same layout)
    Workspace ws;
    PhaseTimer timer;
    struct GraphEntry {
        const double* f;
        int64_t ld_f;
        double* out;
        int64_t ld_out;
        int32_t ndens;
        int64_t launches;
        cudaGraphExec_t exec;
    };
    std::vector<GraphEntry> graphs;  // captured evaluations (VP_FLAG_GRAPH), most recent last
    cudaStream_t cap_stream = nullptr;
    // the correction product runs beside the FMM on a low-priority stream
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    int side_blocks = 0;  // grid of the product beside the FMM: a share of each SM (0: not beside)
    int sms = 152;
    // staging for vp_eval_host
    double* stage = nullptr;
    size_t stage_cap = 0;
    int64_t p2p_pairs = 0;
    int64_t p2p_evals = 0;      // distances evaluated by the symmetric near field
    int64_t last_launches = 0;
    int kernel = VP_KERNEL_LAPLACE;
    DevMH mh;                   // modified-Helmholtz tables (kernel == VP_KERNEL_MHELMHOLTZ)
    int64_t mh_near_ops = 0;    // modelled FP32 operations of its float-float near field
    bool alive = true;

    template <typename T>
    cudaError_t alloc(T** p, size_t n)
    {
        *p = nullptr;
        if (n == 0) n = 1;
        void* q = nullptr;
        cudaError_t e = cudaMalloc(&q, n * sizeof(T));
        if (e != cudaSuccess) return e;
        allocs.push_back(q);
        *p = (T*)q;
        return cudaSuccess;
    }
    template <typename T>
    cudaError_t upload(T** p, const std::vector<T>& h, cudaStream_t s)
    {
        cudaError_t e = alloc(p, h.size());
        if (e != cudaSuccess) return e;
        if (h.empty()) return cudaSuccess;
        return cudaMemcpyAsync(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s);
    }
    ~vp_plan_s()
    {
        for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        if (side) cudaStreamDestroy(side);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        for (void* p : allocs) cudaFree(p);
        if (stage) cudaFree(stage);
        for (auto e : timer.pool) cudaEventDestroy(e);
    }
};

namespace {

vp_status check_plan(vp_plan p)
{
    if (!p || !p->alive) return fail(VP_ERR_STATE, "invalid plan");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device)
        return fail(VP_ERR_STATE, "plan used on a different device than it was created on");
    return VP_OK;
}

int chunk_for(int remaining, int cap)
{
    int nd = 1;
    while (nd * 2 <= remaining && nd * 2 <= cap) nd *= 2;
    return nd;
}

// Integer coordinates of points on the grid 2^-sigma: x 2^sigma is exact in
// float64 (a power of two), rounded to the nearest integer (exact unless
// |x| < 2^(61 - sigma - 53)).
__global__ void k_fix_coords(int64_t n, const double* __restrict__ xy, double scale, long long* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2ll_rn(xy[i] * scale);
}

// sigma with max |coordinate| 2^sigma < 2^61, so that differences stay below 2^62
int fix_sigma(const std::vector<double>& a, const std::vector<double>& b)
{
    double mx = 0.0;
    for (double v : a) mx = std::max(mx, std::fabs(v));
    for (double v : b) mx = std::max(mx, std::fabs(v));
    return mx > 0.0 ? 60 - std::ilogb(mx) : 60;
}

PassGeom forward_geom(vp_plan p)
{
    PassGeom g;
    g.cxy = p->src_xy;
    g.crng = p->box_src;
    g.crho = p->src_rho;
    g.n_charge = (int32_t)p->n_src;
    g.exy = p->tgt_xy;
    g.erng = p->box_tgt;
    g.erho = p->tgt_rho;
    g.n_eval = (int32_t)p->n_tgt;
    g.cfix = p->src_fix;
    g.efix = p->tgt_fix;
    g.fix_sigma = p->fix_sigma;
    g.cpow = p->src_pow;
    g.epow = p->tgt_pow;
    return g;
}

PassGeom adjoint_geom(vp_plan p)
{
    PassGeom g;
    g.cxy = p->tgt_xy;
    g.crng = p->box_tgt;
    g.crho = p->tgt_rho;
    g.n_charge = (int32_t)p->n_tgt;
    g.exy = p->src_xy;
    g.erng = p->box_src;
    g.erho = p->src_rho;
    g.n_eval = (int32_t)p->n_src;
    g.cfix = p->tgt_fix;
    g.efix = p->src_fix;
    g.fix_sigma = p->fix_sigma;
    g.cpow = p->tgt_pow;
    g.epow = p->src_pow;
    return g;
}

// plain float64 reference kernels (VP_FLAG_FP64)
bool use_fp64(vp_plan p) { return p->arith == Arith::kPlain; }
// float-float kernels on the FP32 pipes (VP_FLAG_FF)
bool use_ff(vp_plan p) { return p->arith == Arith::kFF; }

}  // namespace

extern "C" {

const char* vp_status_string(int32_t status)
{
    switch (status) {
        case VP_OK: return "ok";
        case VP_ERR_ARG: return "invalid argument";
        case VP_ERR_CUDA: return "CUDA error";
        case VP_ERR_OOM: return "out of memory";
        case VP_ERR_TIMEOUT: return "device wait timed out";
        case VP_ERR_UNSUPPORTED: return "unsupported option";
        case VP_ERR_STATE: return "invalid plan state";
        default: return "unknown status";
    }
}

const char* vp_last_error(void) { return g_last_error.c_str(); }

const char* vp_version(void) { return "libvp 0.2 sm_103a fp64"; }

}  // extern "C"

namespace {

// One problem's inputs, copied to the host at plan time.
struct ProblemIn {
    int64_t n_src = 0, n_tgt = 0, nnz = 0;
    int64_t n_cols = 0;  // correction columns = density length (n_src, or the p-nodes of an upsampled plan)
    bool has_corr = false;
    std::vector<double> hs, hw, ht;
    std::vector<int64_t> hrow;
    std::vector<int32_t> hcol;
    std::vector<double> hval;
    // the caller's device coordinates (the tree is built from them on the device)
    const double* d_src = nullptr;
    const double* d_tgt = nullptr;
    // the caller's device CSR when its columns and values stay on the device
    const int64_t* d_row = nullptr;
    const int32_t* d_col = nullptr;
    const double* d_val = nullptr;
    bool dev_csr = false;
    double root[3] = {0.0, 0.0, 0.0};
};

// Host arrays of a plan (one problem, or several merged): points in tree
// order, boxes level by level, interaction lists, correction in caller order.
struct Built {
    int64_t n_src = 0, n_tgt = 0, nnz = 0;
    int64_t n_cols = 0;
    bool has_corr = false;
    int n_levels = 0;
    std::vector<double> sxy, txy, ws;
    std::vector<int32_t> src_perm, tgt_perm, sinv, tinv;
    std::vector<double> center, radius, logr;
    std::vector<int32_t> ixy, level, parent, child, is_leaf, brs, brt, leaves, level_start;
    std::vector<int32_t> u_ptr, u_idx, v_ptr, v_idx, w_ptr, w_idx, x_ptr, x_idx;
    std::vector<float> srho, trho, uoff, xoff;
    std::vector<int64_t> hrow;
    std::vector<int32_t> hcol;
    std::vector<double> hval;
    const int64_t* d_row = nullptr;  // caller's device CSR (dev_csr), else hrow/hcol/hval hold it
    const int32_t* d_col = nullptr;
    const double* d_val = nullptr;
    bool dev_csr = false;
    int64_t p2p_pairs = 0;
    double root[3] = {0.0, 0.0, 0.0};
};

// copy_vals: bring the correction's columns and values to the host (plain float64
// plans and forests); otherwise only rowptr is copied and checked here, and the
// columns and values are checked on the device when the plan builds its layout.
vp_status copy_problem(ProblemIn& P, int64_t n_src, const double* src_xy, const double* w, int64_t n_tgt,
                       const double* tgt_xy, const int64_t* corr_rowptr, const int32_t* corr_col,
                       const double* corr_val, int64_t nnz, cudaStream_t s, int64_t n_cols = -1,
                       bool copy_vals = true)
{
    if (n_cols < 0) n_cols = n_src;
    P.n_cols = n_cols;
    if (n_src < 0 || n_tgt < 0 || nnz < 0) return fail(VP_ERR_ARG, "negative size");
    if (n_src > (1LL << 30) || n_tgt > (1LL << 30)) return fail(VP_ERR_ARG, "more than 2^30 points");
    if ((n_src > 0 && (!src_xy || !w)) || (n_tgt > 0 && !tgt_xy)) return fail(VP_ERR_ARG, "NULL point array");
    P.has_corr = corr_rowptr != nullptr;
    if (P.has_corr && nnz > 0 && (!corr_col || !corr_val)) return fail(VP_ERR_ARG, "NULL CSR array");
    if (!P.has_corr && nnz != 0) return fail(VP_ERR_ARG, "nnz > 0 without a CSR");
    P.n_src = n_src;
    P.n_tgt = n_tgt;
    P.nnz = P.has_corr ? nnz : 0;
    P.d_src = src_xy;
    P.d_tgt = tgt_xy;
    P.hs.resize((size_t)n_src * 2);
    P.hw.resize((size_t)n_src);
    P.ht.resize((size_t)n_tgt * 2);
    if (n_src) {
        VP_CUDA(cudaMemcpyAsync(P.hs.data(), src_xy, P.hs.size() * sizeof(double), cudaMemcpyDefault, s));
        VP_CUDA(cudaMemcpyAsync(P.hw.data(), w, P.hw.size() * sizeof(double), cudaMemcpyDefault, s));
    }
    if (n_tgt) VP_CUDA(cudaMemcpyAsync(P.ht.data(), tgt_xy, P.ht.size() * sizeof(double), cudaMemcpyDefault, s));
    if (P.has_corr) {
        P.hrow.resize((size_t)n_tgt + 1);
        VP_CUDA(cudaMemcpyAsync(P.hrow.data(), corr_rowptr, P.hrow.size() * sizeof(int64_t), cudaMemcpyDefault, s));
        P.dev_csr = !copy_vals;
        P.d_row = corr_rowptr;
        P.d_col = corr_col;
        P.d_val = corr_val;
        if (copy_vals) {
            P.hcol.resize((size_t)nnz);
            P.hval.resize((size_t)nnz);
        }
        if (nnz && copy_vals) {
            VP_CUDA(cudaMemcpyAsync(P.hcol.data(), corr_col, P.hcol.size() * sizeof(int32_t), cudaMemcpyDefault, s));
            VP_CUDA(cudaMemcpyAsync(P.hval.data(), corr_val, P.hval.size() * sizeof(double), cudaMemcpyDefault, s));
        }
    }
    VP_CUDA(cudaStreamSynchronize(s));
    if (!finite_all(P.hw)) return fail(VP_ERR_ARG, "non-finite weight");
    if (P.has_corr) {
        if (P.hrow[0] != 0 || P.hrow[(size_t)n_tgt] != nnz) return fail(VP_ERR_ARG, "CSR rowptr does not span [0, nnz]");
        for (int64_t i = 0; i < n_tgt; ++i)
            if (P.hrow[(size_t)i + 1] < P.hrow[(size_t)i]) return fail(VP_ERR_ARG, "CSR rowptr not monotone");
        if (!copy_vals) return VP_OK;
        for (int64_t k = 0; k < nnz; ++k)
            if (P.hcol[(size_t)k] < 0 || P.hcol[(size_t)k] >= n_cols) return fail(VP_ERR_ARG, "CSR column out of range");
        if (!finite_all(P.hval)) return fail(VP_ERR_ARG, "non-finite CSR value");
    }
    return VP_OK;
}

// The tree is built on the device from the caller's coordinates (build_tree_gpu,
// the same tree as the host build_tree).
std::string build_one(ProblemIn& P, const TreeOptions& to, Built& B, cudaStream_t s)
{
    Tree T;
    std::string err = build_tree_gpu(P.n_src, P.d_src, P.n_tgt, P.d_tgt, to, T, s);
    if (!err.empty()) return err;
    const int64_t n_src = P.n_src, n_tgt = P.n_tgt;
    const int32_t nb = (int32_t)T.n_boxes();
    B.n_src = n_src;
    B.n_tgt = n_tgt;
    B.n_cols = P.n_cols;
    B.nnz = P.nnz;
    B.has_corr = P.has_corr;
    B.n_levels = T.n_levels;
    B.root[0] = T.x0;
    B.root[1] = T.y0;
    B.root[2] = T.side;
    B.sxy.resize((size_t)n_src * 2);
    B.txy.resize((size_t)n_tgt * 2);
    B.ws.resize((size_t)n_src);
    B.sinv.resize((size_t)n_src);
    B.tinv.resize((size_t)n_tgt);
    for (int64_t i = 0; i < n_src; ++i) {
        const int32_t c = T.src_perm[(size_t)i];
        B.sxy[2 * i] = P.hs[2 * (size_t)c];
        B.sxy[2 * i + 1] = P.hs[2 * (size_t)c + 1];
        B.ws[(size_t)i] = P.hw[(size_t)c];
        B.sinv[(size_t)c] = (int32_t)i;
    }
    for (int64_t i = 0; i < n_tgt; ++i) {
        const int32_t c = T.tgt_perm[(size_t)i];
        B.txy[2 * i] = P.ht[2 * (size_t)c];
        B.txy[2 * i + 1] = P.ht[2 * (size_t)c + 1];
        B.tinv[(size_t)c] = (int32_t)i;
    }
    B.center.resize((size_t)nb * 2);
    B.radius.resize((size_t)nb);
    B.logr.resize((size_t)nb);
    B.ixy.resize((size_t)nb * 2);
    B.brs.resize((size_t)nb * 2);
    B.brt.resize((size_t)nb * 2);
    for (int32_t b = 0; b < nb; ++b) {
        B.center[2 * (size_t)b] = T.box_cx(b);
        B.center[2 * (size_t)b + 1] = T.box_cy(b);
        B.radius[(size_t)b] = 0.5 * T.box_side(b);
        B.logr[(size_t)b] = std::log(B.radius[(size_t)b]);
        B.ixy[2 * (size_t)b] = T.ix[(size_t)b];
        B.ixy[2 * (size_t)b + 1] = T.iy[(size_t)b];
        B.brs[2 * (size_t)b] = T.src_begin[(size_t)b];
        B.brs[2 * (size_t)b + 1] = T.src_end[(size_t)b];
        B.brt[2 * (size_t)b] = T.tgt_begin[(size_t)b];
        B.brt[2 * (size_t)b + 1] = T.tgt_end[(size_t)b];
        if (T.is_leaf[(size_t)b]) B.leaves.push_back(b);
    }
    for (int32_t b : B.leaves)
        for (int32_t e = T.u_ptr[(size_t)b]; e < T.u_ptr[(size_t)b + 1]; ++e) {
            const int32_t a = T.u_idx[(size_t)e];
            B.p2p_pairs += (int64_t)(T.tgt_end[(size_t)b] - T.tgt_begin[(size_t)b]) *
                           (T.src_end[(size_t)a] - T.src_begin[(size_t)a]);
        }
    B.srho = make_rho(T, B.sxy, true);
    B.trho = make_rho(T, B.txy, false);
    B.uoff = make_list_offsets(T, T.u_ptr, T.u_idx);
    B.xoff = make_list_offsets(T, T.x_ptr, T.x_idx);
    B.src_perm = std::move(T.src_perm);
    B.tgt_perm = std::move(T.tgt_perm);
    B.level = std::move(T.level);
    B.parent = std::move(T.parent);
    B.child = std::move(T.child);
    B.is_leaf = std::move(T.is_leaf);
    B.level_start = std::move(T.level_start);
    B.u_ptr = std::move(T.u_ptr);
    B.u_idx = std::move(T.u_idx);
    B.v_ptr = std::move(T.v_ptr);
    B.v_idx = std::move(T.v_idx);
    B.w_ptr = std::move(T.w_ptr);
    B.w_idx = std::move(T.w_idx);
    B.x_ptr = std::move(T.x_ptr);
    B.x_idx = std::move(T.x_idx);
    B.hrow = std::move(P.hrow);
    B.hcol = std::move(P.hcol);
    B.hval = std::move(P.hval);
    B.d_row = P.d_row;
    B.d_col = P.d_col;
    B.d_val = P.d_val;
    B.dev_csr = P.dev_csr;
    return "";
}

// Several independent problems as one forest: points and caller indices are
// concatenated problem by problem, boxes are reordered level by level (all
// problems' level-l boxes together, so one launch per level serves every
// problem), list entries and ranges are remapped, and the corrections become
// one block-diagonal matrix. Interactions never cross problems.
Built merge(std::vector<Built>& parts)
{
    Built M;
    M.has_corr = false;
    for (const Built& B : parts) {
        M.n_levels = std::max(M.n_levels, B.n_levels);
        M.has_corr = M.has_corr || B.has_corr;
    }
    if (!parts.empty()) std::memcpy(M.root, parts[0].root, sizeof(M.root));
    std::vector<std::vector<int32_t>> newid(parts.size());
    std::vector<int64_t> so(parts.size()), to(parts.size());
    int64_t ns = 0, nt = 0;
    for (size_t k = 0; k < parts.size(); ++k) {
        so[k] = ns;
        to[k] = nt;
        ns += parts[k].n_src;
        nt += parts[k].n_tgt;
        newid[k].assign(parts[k].level.size(), -1);
    }
    M.n_src = ns;
    M.n_cols = ns;
    M.n_tgt = nt;
    int32_t next = 0;
    M.level_start.push_back(0);
    for (int l = 0; l < M.n_levels; ++l) {
        for (size_t k = 0; k < parts.size(); ++k) {
            const Built& B = parts[k];
            if (l >= B.n_levels) continue;
            for (int32_t b = B.level_start[(size_t)l]; b < B.level_start[(size_t)l + 1]; ++b) newid[k][(size_t)b] = next++;
        }
        M.level_start.push_back(next);
    }
    const size_t nb = (size_t)next;
    std::vector<std::pair<int32_t, int32_t>> origin(nb);  // new id -> (problem, old id)
    for (size_t k = 0; k < parts.size(); ++k)
        for (size_t b = 0; b < newid[k].size(); ++b) origin[(size_t)newid[k][b]] = {(int32_t)k, (int32_t)b};
    M.center.resize(nb * 2);
    M.radius.resize(nb);
    M.logr.resize(nb);
    M.ixy.resize(nb * 2);
    M.level.resize(nb);
    M.parent.resize(nb);
    M.child.resize(nb * 4);
    M.is_leaf.resize(nb);
    M.brs.resize(nb * 2);
    M.brt.resize(nb * 2);
    M.u_ptr.assign(nb + 1, 0);
    M.v_ptr.assign(nb + 1, 0);
    M.w_ptr.assign(nb + 1, 0);
    M.x_ptr.assign(nb + 1, 0);
    auto map = [&](size_t k, int32_t b) { return b < 0 ? -1 : newid[k][(size_t)b]; };
    for (size_t n = 0; n < nb; ++n) {
        const size_t k = (size_t)origin[n].first;
        const int32_t b = origin[n].second;
        const Built& B = parts[k];
        M.center[2 * n] = B.center[2 * (size_t)b];
        M.center[2 * n + 1] = B.center[2 * (size_t)b + 1];
        M.radius[n] = B.radius[(size_t)b];
        M.logr[n] = B.logr[(size_t)b];
        M.ixy[2 * n] = B.ixy[2 * (size_t)b];
        M.ixy[2 * n + 1] = B.ixy[2 * (size_t)b + 1];
        M.level[n] = B.level[(size_t)b];
        M.parent[n] = map(k, B.parent[(size_t)b]);
        for (int c = 0; c < 4; ++c) M.child[4 * n + c] = map(k, B.child[4 * (size_t)b + c]);
        M.is_leaf[n] = B.is_leaf[(size_t)b];
        M.brs[2 * n] = B.brs[2 * (size_t)b] + (int32_t)so[k];
        M.brs[2 * n + 1] = B.brs[2 * (size_t)b + 1] + (int32_t)so[k];
        M.brt[2 * n] = B.brt[2 * (size_t)b] + (int32_t)to[k];
        M.brt[2 * n + 1] = B.brt[2 * (size_t)b + 1] + (int32_t)to[k];
        if (M.is_leaf[n]) M.leaves.push_back((int32_t)n);
        auto copy_list = [&](const std::vector<int32_t>& ptr, const std::vector<int32_t>& idx,
                             std::vector<int32_t>& optr, std::vector<int32_t>& oidx, const std::vector<float>* off,
                             std::vector<float>* ooff) {
            for (int32_t e = ptr[(size_t)b]; e < ptr[(size_t)b + 1]; ++e) {
                oidx.push_back(map(k, idx[(size_t)e]));
                if (off) ooff->insert(ooff->end(), off->begin() + 4 * (size_t)e, off->begin() + 4 * (size_t)e + 4);
            }
            optr[n + 1] = (int32_t)oidx.size();
        };
        copy_list(B.u_ptr, B.u_idx, M.u_ptr, M.u_idx, &B.uoff, &M.uoff);
        copy_list(B.v_ptr, B.v_idx, M.v_ptr, M.v_idx, nullptr, nullptr);
        copy_list(B.w_ptr, B.w_idx, M.w_ptr, M.w_idx, nullptr, nullptr);
        copy_list(B.x_ptr, B.x_idx, M.x_ptr, M.x_idx, &B.xoff, &M.xoff);
    }
    int64_t nnz = 0;
    if (M.has_corr) M.hrow.push_back(0);
    for (size_t k = 0; k < parts.size(); ++k) {
        Built& B = parts[k];
        for (double v : B.sxy) M.sxy.push_back(v);
        for (double v : B.txy) M.txy.push_back(v);
        for (double v : B.ws) M.ws.push_back(v);
        for (float v : B.srho) M.srho.push_back(v);
        for (float v : B.trho) M.trho.push_back(v);
        for (int32_t v : B.src_perm) M.src_perm.push_back(v + (int32_t)so[k]);
        for (int32_t v : B.tgt_perm) M.tgt_perm.push_back(v + (int32_t)to[k]);
        for (int32_t v : B.sinv) M.sinv.push_back(v + (int32_t)so[k]);
        for (int32_t v : B.tinv) M.tinv.push_back(v + (int32_t)to[k]);
        M.p2p_pairs += B.p2p_pairs;
        if (M.has_corr) {
            for (int64_t i = 0; i < B.n_tgt; ++i) M.hrow.push_back(nnz + (B.has_corr ? B.hrow[(size_t)i + 1] : 0));
            if (B.has_corr) {
                for (int32_t c : B.hcol) M.hcol.push_back(c + (int32_t)so[k]);
                M.hval.insert(M.hval.end(), B.hval.begin(), B.hval.end());
                nnz += B.nnz;
            }
        }
        B = Built();  // release
    }
    M.nnz = nnz;
    return M;
}

// The grouped correction on the device (vp_csr.cu), from the caller's device CSR or
// (forests) from the host arrays uploaded to temporaries: the columns and values
// are checked on the device, consecutive rows with identical column lists become
// groups (one stored column list each), the values are copied into rows padded to
// even lengths (float64, or hi/lo floats for float-float plans), and for the
// transposed product each column gets the ascending list of the positions where
// it appears among the groups' column lists. Only rowptr, the row flags and the
// groups' column lists pass through the host.
vp_status build_grouped(vp_plan p, Built& B, cudaStream_t s)
{
    const int64_t nrows = B.n_tgt, ncols = B.n_cols, nnz = B.nnz;
    struct Temps {
        std::vector<void*> v;
        ~Temps()
        {
            for (void* q : v) cudaFree(q);
        }
    } tmp;
    auto talloc = [&](size_t bytes) -> void* {
        void* q = nullptr;
        if (cudaMalloc(&q, bytes ? bytes : 1) != cudaSuccess) return nullptr;
        tmp.v.push_back(q);
        return q;
    };
    const int64_t* d_row = B.d_row;
    const int32_t* d_col = B.d_col;
    const double* d_val = B.d_val;
    if (!B.dev_csr) {
        int64_t* r = (int64_t*)talloc(B.hrow.size() * sizeof(int64_t));
        int32_t* c = (int32_t*)talloc(B.hcol.size() * sizeof(int32_t));
        double* v = (double*)talloc(B.hval.size() * sizeof(double));
        if (!r || !c || !v) return fail(VP_ERR_OOM, "device temporaries of the correction");
        VP_CUDA(cudaMemcpyAsync(r, B.hrow.data(), B.hrow.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        if (nnz) {
            VP_CUDA(cudaMemcpyAsync(c, B.hcol.data(), B.hcol.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s));
            VP_CUDA(cudaMemcpyAsync(v, B.hval.data(), B.hval.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        }
        d_row = r;
        d_col = c;
        d_val = v;
    }
    int* d_err = (int*)talloc(sizeof(int));
    uint8_t* d_same = (uint8_t*)talloc((size_t)std::max<int64_t>(nrows, 1));
    if (!d_err || !d_same) return fail(VP_ERR_OOM, "device temporaries of the correction");
    VP_CUDA(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    VP_CUDA(launch_csr_check(nnz, d_col, d_val, ncols, d_err, s));
    VP_CUDA(launch_row_same(nrows, d_row, d_col, d_same, s));
    int herr = 0;
    std::vector<uint8_t> same((size_t)nrows);
    VP_CUDA(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    if (nrows) VP_CUDA(cudaMemcpyAsync(same.data(), d_same, (size_t)nrows, cudaMemcpyDeviceToHost, s));
    VP_CUDA(cudaStreamSynchronize(s));
    if (herr & 1) return fail(VP_ERR_ARG, "CSR column out of range");
    if (herr & 2) return fail(VP_ERR_ARG, "non-finite CSR value");
    // groups of consecutive equal rows, their column offsets, padded value offsets
    std::vector<int32_t> g_r0;
    std::vector<int64_t> g_c0, prow((size_t)nrows + 1, 0);
    int64_t pos = 0;
    int32_t max_m = 0;
    for (int64_t i = 0; i < nrows; ++i) {
        const int64_t len = B.hrow[(size_t)i + 1] - B.hrow[(size_t)i];
        if (i == 0 || !same[(size_t)i]) {
            g_r0.push_back((int32_t)i);
            g_c0.push_back(pos);
            pos += len;
            max_m = std::max<int32_t>(max_m, (int32_t)len);
        }
        prow[(size_t)i + 1] = prow[(size_t)i] + len + (len & 1);
    }
    g_r0.push_back((int32_t)nrows);
    g_c0.push_back(pos);
    DevGroupedCSR& A = p->gfwd;
    int32_t *d_r0 = nullptr, *d_cols = nullptr;
    int64_t *d_c0 = nullptr, *d_prow = nullptr;
    cudaError_t e = p->upload(&d_r0, g_r0, s);
    if (e == cudaSuccess) e = p->upload(&d_c0, g_c0, s);
    if (e == cudaSuccess) e = p->upload(&d_prow, prow, s);
    if (e == cudaSuccess) e = p->alloc(&d_cols, (size_t)pos);
    if (e != cudaSuccess) return cuda_fail(e, "vp_plan_create correction layout");
    A.nrows = (int32_t)nrows;
    A.ngroups = (int32_t)g_r0.size() - 1;
    A.max_m = max_m;
    A.g_r0 = d_r0;
    A.g_c0 = d_c0;
    A.rowptr = d_prow;
    A.cols = d_cols;
    VP_CUDA(launch_group_cols(A.ngroups, d_r0, d_c0, d_row, d_col, d_cols, s));
    if (p->arith == Arith::kF64) {
        int2* vi = nullptr;
        int32_t* vexp = nullptr;
        VP_CUDA(p->alloc(&vi, (size_t)prow[(size_t)nrows]));
        VP_CUDA(p->alloc(&vexp, (size_t)std::max<int64_t>(nrows, 1)));
        VP_CUDA(launch_fix_values(nrows, d_row, d_prow, d_val, vi, vexp, s));
        A.vi = vi;
        A.vexp = vexp;
    } else {
        float2* vf = nullptr;
        VP_CUDA(p->alloc(&vf, (size_t)prow[(size_t)nrows]));
        VP_CUDA(launch_pad_values(nrows, d_row, d_prow, d_val, vf, s));
        A.vf = vf;
    }
    // positions of every column among the groups' column lists, ascending
    std::vector<int32_t> hcols((size_t)pos);
    if (pos) VP_CUDA(cudaMemcpyAsync(hcols.data(), d_cols, (size_t)pos * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    VP_CUDA(cudaStreamSynchronize(s));
    std::vector<int64_t> inc_ptr((size_t)ncols + 1, 0), inc_pos((size_t)pos);
    for (int64_t q = 0; q < pos; ++q) inc_ptr[(size_t)hcols[(size_t)q] + 1]++;
    for (int64_t c = 0; c < ncols; ++c) inc_ptr[(size_t)c + 1] += inc_ptr[(size_t)c];
    {
        std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
        for (int64_t q = 0; q < pos; ++q) inc_pos[(size_t)fill[(size_t)hcols[(size_t)q]]++] = q;
    }
    int64_t *d_iptr = nullptr, *d_ipos = nullptr;
    e = p->upload(&d_iptr, inc_ptr, s);
    if (e == cudaSuccess) e = p->upload(&d_ipos, inc_pos, s);
    if (e == cudaSuccess) e = p->alloc(&p->ws.adj_partial, (size_t)pos * p->nd_cap);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // before the temporaries are freed
    if (e != cudaSuccess) return cuda_fail(e, "vp_plan_create correction layout");
    A.adj_ncols = ncols;
    A.inc_ptr = d_iptr;
    A.inc_pos = d_ipos;
    return VP_OK;
}

vp_status finalize(vp_plan p, Built& B, int P, cudaStream_t s)
{
    const int64_t n_src = B.n_src, n_tgt = B.n_tgt, nnz = B.nnz, n_cols = B.n_cols;
    const bool has_corr = B.has_corr;
    const int32_t nb = (int32_t)B.level.size();
    p->n_src = n_src;
    p->n_f = n_cols;
    p->n_tgt = n_tgt;
    p->nnz = has_corr ? nnz : 0;
    p->p2p_pairs = B.p2p_pairs;
    p->stat_levels = B.n_levels;
    p->stat_boxes = nb;
    p->stat_leaves = (int64_t)B.leaves.size();
    p->stat_u = 0;
    p->stat_w = 0;
    for (int32_t b : B.leaves) {
        p->stat_u += B.u_ptr[(size_t)b + 1] - B.u_ptr[(size_t)b];
        p->stat_w += B.w_ptr[(size_t)b + 1] - B.w_ptr[(size_t)b];
    }
    p->stat_v = (int64_t)B.v_idx.size();
    p->stat_x = (int64_t)B.x_idx.size();
    std::memcpy(p->stat_root, B.root, sizeof(p->stat_root));

    // transposed correction (columns = sources), for the adjoint of plain float64 plans
    // (the grouped plans compute Pi^T g from the forward layout, see vp_csr.cu)
    std::vector<int64_t> hcptr;
    std::vector<int32_t> hcrow;
    std::vector<double> hcval;
    if (has_corr && p->arith == Arith::kPlain) {
        hcptr.assign((size_t)n_cols + 1, 0);
        for (int64_t k = 0; k < nnz; ++k) hcptr[(size_t)B.hcol[(size_t)k] + 1]++;
        for (int64_t j = 0; j < n_cols; ++j) hcptr[(size_t)j + 1] += hcptr[(size_t)j];
        std::vector<int64_t> fill(hcptr.begin(), hcptr.end() - 1);
        hcrow.resize((size_t)nnz);
        hcval.resize((size_t)nnz);
        for (int64_t i = 0; i < n_tgt; ++i)
            for (int64_t k = B.hrow[(size_t)i]; k < B.hrow[(size_t)i + 1]; ++k) {
                const int64_t pos = fill[(size_t)B.hcol[(size_t)k]]++;
                hcrow[(size_t)pos] = (int32_t)i;
                hcval[(size_t)pos] = B.hval[(size_t)k];
            }
    }
    size_t off[7];
    std::vector<double> tables = make_tables(P, off);
    std::vector<float> logtab = make_log_table();
    std::vector<double2> log64;
    std::vector<double> elog64;
    make_log64_tables(log64, elog64);
    size_t offf[8];
    std::vector<float> fftab = make_ff_tables(P, offf);

    cudaError_t e = cudaSuccess;
    auto up = [&](auto** dst, const auto& h) {
        if (e == cudaSuccess) e = p->upload(dst, h, s);
    };
    double* d_xy_s = nullptr;
    double* d_xy_t = nullptr;
    up(&d_xy_s, B.sxy);
    up(&d_xy_t, B.txy);
    p->src_xy = (double2*)d_xy_s;
    p->tgt_xy = (double2*)d_xy_t;
    p->fix_sigma = fix_sigma(B.sxy, B.txy);
    {
        long long *fs = nullptr, *ft = nullptr;
        if (e == cudaSuccess) e = p->alloc(&fs, B.sxy.size());
        if (e == cudaSuccess) e = p->alloc(&ft, B.txy.size());
        const double scale = std::ldexp(1.0, p->fix_sigma);
        if (e == cudaSuccess && !B.sxy.empty())
            k_fix_coords<<<(int)std::min<size_t>((B.sxy.size() + 255) / 256, 4096), 256, 0, s>>>(
                (int64_t)B.sxy.size(), d_xy_s, scale, fs);
        if (e == cudaSuccess && !B.txy.empty())
            k_fix_coords<<<(int)std::min<size_t>((B.txy.size() + 255) / 256, 4096), 256, 0, s>>>(
                (int64_t)B.txy.size(), d_xy_t, scale, ft);
        if (e == cudaSuccess) e = cudaGetLastError();
        p->src_fix = (longlong2*)fs;
        p->tgt_fix = (longlong2*)ft;
    }
    up(&p->w_sorted, B.ws);
    up(&p->src_perm, B.src_perm);
    up(&p->tgt_perm, B.tgt_perm);
    up(&p->src_inv, B.sinv);
    up(&p->tgt_inv, B.tinv);
    up(&p->box_src, B.brs);
    up(&p->box_tgt, B.brt);
    double *d_center = nullptr, *d_radius = nullptr, *d_logr = nullptr, *d_tab = nullptr;
    int32_t *d_ixy = nullptr, *d_parent = nullptr, *d_child = nullptr, *d_leaf = nullptr, *d_leaves = nullptr;
    int32_t *d_up = nullptr, *d_ui = nullptr, *d_vp = nullptr, *d_vi = nullptr, *d_wp = nullptr, *d_wi = nullptr,
            *d_xp = nullptr, *d_xi = nullptr;
    up(&d_center, B.center);
    up(&d_radius, B.radius);
    up(&d_logr, B.logr);
    up(&d_ixy, B.ixy);
    up(&d_parent, B.parent);
    up(&d_child, B.child);
    up(&d_leaf, B.is_leaf);
    {
        // costliest leaves first, so the persistent near-field kernel ends evenly
        std::vector<int64_t> cost(B.leaves.size());
        for (size_t i = 0; i < B.leaves.size(); ++i) {
            const int32_t b = B.leaves[i];
            int64_t srcs = 0;
            for (int32_t e2 = B.u_ptr[(size_t)b]; e2 < B.u_ptr[(size_t)b + 1]; ++e2) {
                const int32_t a = B.u_idx[(size_t)e2];
                srcs += B.brs[2 * (size_t)a + 1] - B.brs[2 * (size_t)a];
            }
            cost[i] = (int64_t)(B.brt[2 * (size_t)b + 1] - B.brt[2 * (size_t)b]) * srcs;
        }
        std::vector<size_t> order(B.leaves.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b2) { return cost[a] > cost[b2]; });
        std::vector<int32_t> sorted(order.size());
        for (size_t i = 0; i < order.size(); ++i) sorted[i] = B.leaves[order[i]];
        B.leaves.swap(sorted);
    }
    up(&d_leaves, B.leaves);
    // symmetric near field when the charge points of both passes are the evaluation
    // points (same coordinates, same tree order) and the U lists are symmetric
    // (the modified-Helmholtz kernel has a symmetric form on its float-float path only)
    const bool sym_kernel = p->kernel == VP_KERNEL_LAPLACE ? p->arith != Arith::kPlain : p->arith == Arith::kFF;
    bool sym = sym_kernel && n_src == n_tgt && n_src > 0 && B.sxy == B.txy && B.brs == B.brt;
    if (sym) {
        for (int32_t b : B.leaves) {
            for (int32_t e2 = B.u_ptr[(size_t)b]; e2 < B.u_ptr[(size_t)b + 1] && sym; ++e2) {
                const int32_t a = B.u_idx[(size_t)e2];
                if (a == b) continue;
                bool found = false;
                for (int32_t f = B.u_ptr[(size_t)a]; f < B.u_ptr[(size_t)a + 1]; ++f)
                    if (B.u_idx[(size_t)f] == b) found = true;
                sym = found;
            }
            if (!sym) break;
        }
    }
    std::vector<int32_t> sym_leaves, in_ptr, in_pptr, in_pbox, own;
    std::vector<int64_t> sym_off, in_slot;
    int64_t nslots = 0;
    if (sym) {
        sym_off.assign(B.u_idx.size(), -1);
        std::vector<std::vector<int64_t>> rin((size_t)nb);
        std::vector<std::vector<int32_t>> rbox((size_t)nb);
        std::vector<int32_t> asc(B.leaves);
        std::sort(asc.begin(), asc.end());
        std::vector<int64_t> cost((size_t)nb, 0);
        own.assign((size_t)nb, 0);
        for (int32_t b : asc) {
            const int64_t nt_b = B.brt[2 * (size_t)b + 1] - B.brt[2 * (size_t)b];
            if (nt_b == 0) continue;
            const int64_t ng = (nt_b + 31) / 32;
            // own pairs once each when the leaf is small enough and no two of its
            // points coincide (the coincident-pair bookkeeping stays directed)
            // (float-float Laplace kernel only; the float64 kernel sums a leaf's own pairs directed)
            bool own_ok = ng <= kOwnGroups && p->kernel == VP_KERNEL_LAPLACE && p->arith == Arith::kFF;
            if (own_ok) {
                std::vector<std::pair<double, double>> pts;
                for (int32_t j = B.brt[2 * (size_t)b]; j < B.brt[2 * (size_t)b + 1]; ++j)
                    pts.emplace_back(B.txy[2 * (size_t)j], B.txy[2 * (size_t)j + 1]);
                std::sort(pts.begin(), pts.end());
                for (size_t k = 1; k < pts.size() && own_ok; ++k) own_ok = !(pts[k] == pts[k - 1]);
            }
            own[(size_t)b] = own_ok ? 1 : 0;
            int64_t work = 0, own_cost = 0;
            for (int32_t e2 = B.u_ptr[(size_t)b]; e2 < B.u_ptr[(size_t)b + 1]; ++e2) {
                const int32_t a = B.u_idx[(size_t)e2];
                const int64_t na = B.brs[2 * (size_t)a + 1] - B.brs[2 * (size_t)a];
                if (a < b || na == 0) continue;
                if (a == b) {
                    work += own_ok ? 0 : na;
                    if (own_ok) {
                        // distances evaluated for the leaf's own pairs: each pair inside a
                        // group of 32 and between groups of different passes of 64 targets
                        // once, pairs between the two groups of one pass in both directions
                        int64_t ev = 0;
                        for (int64_t g1 = 0; g1 < ng; ++g1) {
                            const int64_t s1 = std::min<int64_t>(32, nt_b - 32 * g1);
                            ev += s1 * (s1 - 1) / 2;
                            for (int64_t g2 = g1 + 1; g2 < ng; ++g2) {
                                const int64_t s2 = std::min<int64_t>(32, nt_b - 32 * g2);
                                ev += (g1 / 2 == g2 / 2) ? 2 * s1 * s2 : s1 * s2;
                            }
                        }
                        p->p2p_evals += ev;
                        own_cost = ev;
                    }
                    continue;
                }
                work += na;
                sym_off[(size_t)e2] = nslots;
                for (int64_t gi = 0; gi < ng; ++gi) rin[(size_t)a].push_back(nslots + gi * na);
                rbox[(size_t)a].push_back(b);
                nslots += ng * na;
            }
            cost[(size_t)b] = nt_b * work + own_cost;
            p->p2p_evals += nt_b * work;
        }
        sym_leaves = B.leaves;
        std::stable_sort(sym_leaves.begin(), sym_leaves.end(),
                         [&](int32_t a, int32_t b2) { return cost[(size_t)a] > cost[(size_t)b2]; });
        in_ptr.assign((size_t)nb + 1, 0);
        in_pptr.assign((size_t)nb + 1, 0);
        for (int32_t a = 0; a < nb; ++a) {
            in_ptr[(size_t)a + 1] = in_ptr[(size_t)a] + (int32_t)rin[(size_t)a].size();
            in_pptr[(size_t)a + 1] = in_pptr[(size_t)a] + (int32_t)rbox[(size_t)a].size();
            in_slot.insert(in_slot.end(), rin[(size_t)a].begin(), rin[(size_t)a].end());
            in_pbox.insert(in_pbox.end(), rbox[(size_t)a].begin(), rbox[(size_t)a].end());
        }
    }
    std::vector<int32_t> pt_leaf;
    if (sym) {
        pt_leaf.assign((size_t)n_tgt, 0);
        for (int32_t b : B.leaves)
            for (int32_t j = B.brt[2 * (size_t)b]; j < B.brt[2 * (size_t)b + 1]; ++j) pt_leaf[(size_t)j] = b;
    }
    int32_t *d_sym_leaves = nullptr, *d_in_ptr = nullptr, *d_in_pptr = nullptr, *d_in_pbox = nullptr,
            *d_pt_leaf = nullptr, *d_own = nullptr;
    int64_t *d_sym_off = nullptr, *d_in_slot = nullptr;
    if (sym) {
        up(&d_sym_leaves, sym_leaves);
        up(&d_sym_off, sym_off);
        up(&d_in_ptr, in_ptr);
        up(&d_in_slot, in_slot);
        up(&d_in_pptr, in_pptr);
        up(&d_in_pbox, in_pbox);
        up(&d_pt_leaf, pt_leaf);
        up(&d_own, own);
    }
    up(&d_up, B.u_ptr);
    up(&d_ui, B.u_idx);
    up(&d_vp, B.v_ptr);
    up(&d_vi, B.v_idx);
    up(&d_wp, B.w_ptr);
    up(&d_wi, B.w_idx);
    up(&d_xp, B.x_ptr);
    up(&d_xi, B.x_idx);
    up(&d_tab, tables);
    float *d_logtab = nullptr, *d_srho = nullptr, *d_trho = nullptr, *d_fftab = nullptr;
    int32_t* d_level = nullptr;
    up(&d_logtab, logtab);
    double2* d_log64 = nullptr;
    double* d_elog64 = nullptr;
    double2* d_m2m64 = nullptr;
    up(&d_log64, log64);
    up(&d_elog64, elog64);
    up(&d_m2m64, make_m2m64_table(P));
    double2* d_l2l64 = nullptr;
    up(&d_l2l64, make_l2l64_table(P));
    std::vector<uint16_t> m2lh;
    std::vector<int32_t> m2le;
    std::vector<double2> mtpow_s;
    std::vector<double> tau_pow;
    make_m2l_tensor_tables(P, m2lh, m2le, mtpow_s, tau_pow);
    uint16_t* d_m2lh = nullptr;
    int32_t* d_m2le = nullptr;
    double2* d_mtpow_s = nullptr;
    double* d_tau_pow = nullptr;
    up(&d_m2lh, m2lh);
    up(&d_m2le, m2le);
    up(&d_mtpow_s, mtpow_s);
    up(&d_tau_pow, tau_pow);
    longlong2* d_logint = nullptr;
    up(&d_logint, make_logint_table());
    up(&d_fftab, fftab);
    up(&d_srho, B.srho);
    up(&d_trho, B.trho);
    up(&d_level, B.level);
    float *d_uoff = nullptr, *d_xoff = nullptr;
    up(&d_uoff, B.uoff);
    up(&d_xoff, B.xoff);
    p->src_rho = (float4*)d_srho;
    p->tgt_rho = (float4*)d_trho;
    p->grouped = has_corr && p->arith != Arith::kPlain;
    if (has_corr && !p->grouped) {
        up(&p->rowptr, B.hrow);
        up(&p->col, B.hcol);
        up(&p->val, B.hval);
        up(&p->cptr, hcptr);
        up(&p->crow, hcrow);
        up(&p->cval, hcval);
    }
    if (p->grouped && e == cudaSuccess) {
        const vp_status gst = build_grouped(p, B, s);
        if (gst != VP_OK) return gst;
    }
    const int P1 = P + 1;
    const int64_t npts = std::max<int64_t>(std::max<int64_t>(std::max<int64_t>(n_src, n_tgt), n_cols), 1);
    if (e == cudaSuccess) e = p->alloc(&p->ws.q, (size_t)npts * p->nd_cap);
    if (e == cudaSuccess) e = p->alloc(&p->ws.qf, (size_t)npts * p->nd_cap);
    if (e == cudaSuccess) e = p->alloc(&p->ws.psi, (size_t)npts * 2 * p->nd_cap);
    if (e == cudaSuccess) e = p->alloc(&p->ws.xf, (size_t)npts * p->nd_cap);
    if (e == cudaSuccess) e = p->alloc(&p->ws.M, (size_t)nb * P1 * p->nd_cap);
    if (e == cudaSuccess) e = p->alloc(&p->ws.Mf, (size_t)nb * P1 * p->nd_cap);
    if (e == cudaSuccess) e = p->alloc(&p->ws.Lf, (size_t)nb * P1 * p->nd_cap);
    if (e == cudaSuccess) e = p->alloc(&p->ws.L, (size_t)nb * P1 * p->nd_cap);
    if (e == cudaSuccess) e = p->alloc(&p->ws.work, 4);
    if (e == cudaSuccess && p->grouped) {
        int least = 0, greatest = 0;
        e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, least);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device);
        p->side_blocks = 0;  // the product after the FMM until vp_plan_set_overlap asks otherwise
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = p->alloc(&p->ws.m2m_count, (size_t)std::max<int32_t>(nb, 1));
    if (e == cudaSuccess) e = cudaMemsetAsync(p->ws.m2m_count, 0, sizeof(int) * (size_t)std::max<int32_t>(nb, 1), s);
    if (e == cudaSuccess && sym) e = p->alloc(&p->ws.slots, (size_t)std::max<int64_t>(nslots, 1) * p->nd_cap);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "vp_plan_create upload");
    p->ws.nd_cap = p->nd_cap;

    DevTree& dt = p->dt;
    dt.nbox = nb;
    dt.nlevels = B.n_levels;
    dt.nleaf = (int32_t)B.leaves.size();
    dt.center = (const double2*)d_center;
    dt.radius = d_radius;
    dt.log_radius = d_logr;
    dt.ixy = d_ixy;
    dt.level = d_level;
    dt.parent = d_parent;
    dt.child = d_child;
    dt.is_leaf = d_leaf;
    dt.src_rng = p->box_src;
    dt.tgt_rng = p->box_tgt;
    dt.leaves = d_leaves;
    dt.u_ptr = d_up;
    dt.u_idx = d_ui;
    dt.u_off = (const float4*)d_uoff;
    dt.x_off = (const float4*)d_xoff;
    dt.v_ptr = d_vp;
    dt.v_idx = d_vi;
    dt.w_ptr = d_wp;
    dt.w_idx = d_wi;
    dt.x_ptr = d_xp;
    dt.x_idx = d_xi;
    dt.level_start = B.level_start;
    dt.sym = sym;
    dt.sym_leaves = d_sym_leaves;
    dt.sym_off = d_sym_off;
    dt.sym_in_ptr = d_in_ptr;
    dt.sym_in_slot = d_in_slot;
    dt.sym_in_pptr = d_in_pptr;
    dt.sym_in_pbox = d_in_pbox;
    dt.sym_pt_leaf = d_pt_leaf;
    dt.sym_own = d_own;
    dt.sym_slots = nslots;
    if (p->arith == Arith::kF64) {
        // the points' powers in their leaves (P2M and L2P inputs of the float64 kernels)
        cudaError_t ep = p->alloc(&p->src_pow, (size_t)n_src * P);
        if (ep == cudaSuccess) ep = p->alloc(&p->tgt_pow, (size_t)n_tgt * P);
        if (ep == cudaSuccess && n_src > 0) ep = launch_point_powers(P, dt, p->box_src, p->src_xy, p->src_pow, s);
        if (ep == cudaSuccess && n_tgt > 0) ep = launch_point_powers(P, dt, p->box_tgt, p->tgt_xy, p->tgt_pow, s);
        if (ep != cudaSuccess) return cuda_fail(ep, "vp_plan_create point powers");
    }
    DevTables& tb = p->tab;
    tb.H = d_tab + off[0];
    tb.Bm = d_tab + off[1];
    tb.Bl = d_tab + off[2];
    tb.tpow = (const double2*)(d_tab + off[3]);
    tb.mtpow = (const double2*)(d_tab + off[4]);
    tb.log2o = d_tab + off[5];
    tb.zpow = (const double2*)(d_tab + off[6]);
    tb.logtab = (const float4*)d_logtab;
    tb.log64 = d_log64;
    tb.elog64 = d_elog64;
    tb.m2m64 = d_m2m64;
    tb.l2l64 = d_l2l64;
    tb.m2lh = reinterpret_cast<const uint32_t*>(d_m2lh);
    tb.m2le = d_m2le;
    tb.mtpow_s = d_mtpow_s;
    tb.tau_pow = d_tau_pow;
    tb.logint = d_logint;
    tb.Hf = (const float2*)(d_fftab + offf[0]);
    tb.tpowf = (const float4*)(d_fftab + offf[1]);
    tb.mtpowf = (const float4*)(d_fftab + offf[2]);
    tb.log2of = (const float2*)(d_fftab + offf[3]);
    tb.invlf = (const float2*)(d_fftab + offf[4]);
    tb.Bmf = (const float2*)(d_fftab + offf[5]);
    tb.Blf = (const float2*)(d_fftab + offf[6]);
    tb.zpowf = (const float2*)(d_fftab + offf[7]);
    const void* vec16[] = {tb.tpow, tb.mtpow, tb.zpow, tb.logtab, tb.tpowf, tb.mtpowf, p->src_xy, p->tgt_xy,
                           p->src_rho, p->tgt_rho, p->ws.M, p->ws.Mf, p->ws.L, p->ws.Lf, p->dt.u_off, p->dt.x_off,
                           tb.log64, p->gfwd.vi, tb.m2lh, tb.mtpow_s, p->src_fix, p->tgt_fix, tb.logint};
    const void* vec8[] = {tb.Hf, tb.log2of, tb.invlf, tb.Bmf, tb.Blf, tb.zpowf, p->ws.qf, p->ws.xf, p->gfwd.vf};
    bool ok = true;
    for (const void* q : vec16) ok = ok && ((uintptr_t)q % 16 == 0);
    for (const void* q : vec8) ok = ok && ((uintptr_t)q % 8 == 0);
    if (!ok) return fail(VP_ERR_CUDA, "internal error: misaligned device table");
    return VP_OK;
}

vp_status plan_options(const vp_options* opt_in, vp_options& opt, int& P, int& leaf, int& max_level, int& max_dens)
{
    std::memset(&opt, 0, sizeof(opt));
    if (opt_in) opt = *opt_in;
    P = opt.p_fmm == 0 ? 30 : opt.p_fmm;
    if (!p_supported(P)) return fail(VP_ERR_UNSUPPORTED, "p_fmm must be 16, 24 or 30");
    leaf = opt.leaf == 0 ? 64 : opt.leaf;
    max_level = opt.max_level == 0 ? 24 : opt.max_level;
    max_dens = opt.max_dens <= 0 ? 1 : opt.max_dens;
    if (leaf < 1 || leaf > 4096) return fail(VP_ERR_ARG, "leaf outside [1, 4096]");
    if (max_level < 1 || max_level >= kCoordBits) return fail(VP_ERR_ARG, "max_level outside [1, 27]");
    if (opt.kernel != VP_KERNEL_LAPLACE && opt.kernel != VP_KERNEL_MHELMHOLTZ)
        return fail(VP_ERR_ARG, "unknown kernel");
    if (opt.kernel == VP_KERNEL_MHELMHOLTZ && !(opt.lambda > 0.0 && std::isfinite(opt.lambda)))
        return fail(VP_ERR_ARG, "the modified-Helmholtz kernel needs a finite lambda > 0");
    if ((opt.flags & VP_FLAG_FF) && (opt.flags & VP_FLAG_FP64))
        return fail(VP_ERR_ARG, "VP_FLAG_FF and VP_FLAG_FP64 exclude each other");
    return VP_OK;
}

// Operator tables of the modified-Helmholtz kernel for the plan's tree: one
// half side per level (a single tree: every box of a level has the same size)
// and a bound on every near-field distance.
vp_status setup_mh(vp_plan p, const Built& B, double lambda, cudaStream_t s)
{
    const int nl = B.n_levels;
    std::vector<double> R((size_t)std::max(nl, 1), 0.0);
    for (size_t b = 0; b < B.level.size(); ++b) {
        double& r = R[(size_t)B.level[b]];
        if (r == 0.0) r = B.radius[b];
        else if (r != B.radius[b]) return fail(VP_ERR_UNSUPPORTED, "modified-Helmholtz plans need one tree");
    }
    for (int l = 1; l < nl; ++l)
        if (R[(size_t)l] == 0.0) R[(size_t)l] = 0.5 * R[(size_t)l - 1];
    std::vector<double> dmax(B.level.size(), 0.0);
    for (int32_t b : B.leaves)
        for (int32_t e = B.u_ptr[(size_t)b]; e < B.u_ptr[(size_t)b + 1]; ++e) {
            const int32_t a = B.u_idx[(size_t)e];
            const double dx = B.center[2 * (size_t)a] - B.center[2 * (size_t)b];
            const double dy = B.center[2 * (size_t)a + 1] - B.center[2 * (size_t)b + 1];
            dmax[(size_t)b] = std::max(dmax[(size_t)b], std::sqrt(dx * dx + dy * dy) +
                                                           std::sqrt(2.0) * (B.radius[(size_t)a] + B.radius[(size_t)b]));
        }
    MhTables T;
    const std::string err = make_mh_tables(p->P, lambda, R, dmax, use_ff(p), T);
    if (!err.empty()) return fail(VP_ERR_ARG, err);
    // FP32 operations of the float-float near field per evaluation (one density):
    // per evaluated distance about 92 + 2 (deg - m + 1) + 24 m (distance, table log,
    // T, FP32 tails, float-float heads, K0, accumulate) for the leaf's (deg, m), +14
    // when the evaluation serves both directions (symmetric near field)
    p->mh_near_ops = 0;
    for (int32_t b : B.leaves) {
        int64_t own = 0, both = 0;
        for (int32_t e2 = B.u_ptr[(size_t)b]; e2 < B.u_ptr[(size_t)b + 1]; ++e2) {
            const int32_t a = B.u_idx[(size_t)e2];
            const int64_t na = B.brs[2 * (size_t)a + 1] - B.brs[2 * (size_t)a];
            if (!p->dt.sym || a == b) own += na;
            else if (a > b) both += na;
        }
        const int code = T.leaf_deg[(size_t)b], deg = code & 0xff, m = code >> 8;
        const int64_t ops = 92 + 2 * (deg - m + 1) + 24 * m;
        p->mh_near_ops += (int64_t)(B.brt[2 * (size_t)b + 1] - B.brt[2 * (size_t)b]) * (own * ops + both * (ops + 14));
    }
    cudaError_t e = cudaSuccess;
    double *d_spow = nullptr, *d_na = nullptr, *d_nb = nullptr;
    double2 *d_tm = nullptr, *d_tl = nullptr, *d_tv = nullptr;
    float4* d_tvf = nullptr;
    int32_t* d_deg = nullptr;
    if (e == cudaSuccess) e = p->upload(&d_deg, T.leaf_deg, s);
    if (e == cudaSuccess) e = p->upload(&d_spow, T.spow, s);
    if (e == cudaSuccess) e = p->upload(&d_na, T.near_a, s);
    if (e == cudaSuccess) e = p->upload(&d_nb, T.near_b, s);
    if (e == cudaSuccess) e = p->upload(&d_tm, T.Tm, s);
    if (e == cudaSuccess) e = p->upload(&d_tl, T.Tl, s);
    if (e == cudaSuccess && !T.Tv.empty()) e = p->upload(&d_tv, T.Tv, s);
    if (e == cudaSuccess && !T.Tvf.empty()) e = p->upload(&d_tvf, T.Tvf, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "vp_plan_create upload");
    DevMH& m = p->mh;
    m.lambda = lambda;
    m.lam2_4 = 0.25 * lambda * lambda;
    m.c0 = std::log(0.5 * lambda) + 0.577215664901532860606512090082402431;
    m.psi_scale = -lambda * lambda;
    m.inv_fact_P = T.inv_fact_P;
    m.near_deg = T.near_deg;
    m.leaf_deg = d_deg;
    m.near_a = d_na;
    m.near_b = d_nb;
    m.spow = d_spow;
    m.Tm = d_tm;
    m.Tl = d_tl;
    m.Tv = d_tv;
    m.Tvf = d_tvf;
    return VP_OK;
}

vp_plan new_plan(const vp_options& opt, int P, int leaf, int max_dens)
{
    vp_plan p = new (std::nothrow) vp_plan_s();
    if (!p) return nullptr;
    cudaGetDevice(&p->device);
    p->P = P;
    p->leaf = leaf;
    p->max_dens = max_dens;
    p->kernel = opt.kernel;
    p->nd_cap = opt.kernel == VP_KERNEL_MHELMHOLTZ ? 1 : chunk_for(max_dens, 8);
    p->flags = (uint32_t)opt.flags;
    p->arith = (p->flags & VP_FLAG_FF) ? Arith::kFF : (p->flags & VP_FLAG_FP64) ? Arith::kPlain : Arith::kF64;
    p->timer.on = (p->flags & VP_FLAG_TIMING) != 0;
    return p;
}

}  // namespace

extern "C" {

vp_status vp_plan_create(vp_plan* out, int64_t n_src, const double* src_xy, const double* w, int64_t n_tgt,
                         const double* tgt_xy, const int64_t* corr_rowptr, const int32_t* corr_col,
                         const double* corr_val, int64_t nnz, const vp_options* opt_in, void* stream)
{
    g_last_error.clear();
    if (!out) return fail(VP_ERR_ARG, "out is NULL");
    *out = nullptr;
    vp_options opt;
    int P, leaf, max_level, max_dens;
    vp_status st = plan_options(opt_in, opt, P, leaf, max_level, max_dens);
    if (st != VP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    ProblemIn in;
    st = copy_problem(in, n_src, src_xy, w, n_tgt, tgt_xy, corr_rowptr, corr_col, corr_val, nnz, s, -1,
                      (opt.flags & VP_FLAG_FP64) != 0);
    if (st != VP_OK) return st;
    TreeOptions to;
    to.leaf = leaf;
    to.max_level = max_level;
    std::memcpy(to.root, opt.root, sizeof(to.root));
    Built B;
    std::string err = build_one(in, to, B, s);
    if (!err.empty()) return fail(VP_ERR_ARG, err);
    vp_plan p = new_plan(opt, P, leaf, max_dens);
    if (!p) return fail(VP_ERR_OOM, "host allocation");
    st = finalize(p, B, P, s);
    if (st == VP_OK && p->kernel == VP_KERNEL_MHELMHOLTZ) st = setup_mh(p, B, opt.lambda, s);
    if (st != VP_OK) {
        delete p;
        return st;
    }
    *out = p;
    return VP_OK;
}

vp_status vp_plan_create_many(vp_plan* out, int32_t nprob, const int64_t* n_src, const double* const* src_xy,
                              const double* const* w, const int64_t* n_tgt, const double* const* tgt_xy,
                              const int64_t* const* corr_rowptr, const int32_t* const* corr_col,
                              const double* const* corr_val, const int64_t* nnz, const double* roots,
                              const vp_options* opt_in, void* stream)
{
    g_last_error.clear();
    if (!out) return fail(VP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nprob < 1) return fail(VP_ERR_ARG, "nprob < 1");
    if (!n_src || !src_xy || !w || !n_tgt || !tgt_xy) return fail(VP_ERR_ARG, "NULL per-problem array");
    vp_options opt;
    int P, leaf, max_level, max_dens;
    vp_status st = plan_options(opt_in, opt, P, leaf, max_level, max_dens);
    if (st != VP_OK) return st;
    if (opt.kernel != VP_KERNEL_LAPLACE)
        return fail(VP_ERR_UNSUPPORTED, "the modified-Helmholtz kernel is available through vp_plan_create only");
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<Built> parts((size_t)nprob);
    int64_t tot_s = 0, tot_t = 0;
    for (int32_t k = 0; k < nprob; ++k) {
        ProblemIn in;
        st = copy_problem(in, n_src[k], src_xy[k], w[k], n_tgt[k], tgt_xy[k], corr_rowptr ? corr_rowptr[k] : nullptr,
                          corr_col ? corr_col[k] : nullptr, corr_val ? corr_val[k] : nullptr, nnz ? nnz[k] : 0, s);
        if (st != VP_OK) return fail(st, "problem " + std::to_string(k) + ": " + g_last_error);
        tot_s += n_src[k];
        tot_t += n_tgt[k];
        if (tot_s > (1LL << 30) || tot_t > (1LL << 30)) return fail(VP_ERR_ARG, "more than 2^30 points in total");
        TreeOptions to;
        to.leaf = leaf;
        to.max_level = max_level;
        if (roots) std::memcpy(to.root, roots + 3 * (size_t)k, sizeof(to.root));
        std::string err = build_one(in, to, parts[(size_t)k], s);
        if (!err.empty()) return fail(VP_ERR_ARG, "problem " + std::to_string(k) + ": " + err);
    }
    Built B = merge(parts);
    vp_plan p = new_plan(opt, P, leaf, max_dens);
    if (!p) return fail(VP_ERR_OOM, "host allocation");
    p->n_problems = nprob;
    st = finalize(p, B, P, s);
    if (st != VP_OK) {
        delete p;
        return st;
    }
    *out = p;
    return VP_OK;
}

vp_status vp_plan_create_upsampled(vp_plan* out, int64_t n_src, const double* src_xy, const double* w,
                                   int64_t n_tgt, const double* tgt_xy, const int64_t* corr_rowptr,
                                   const int32_t* corr_col, const double* corr_val, int64_t nnz,
                                   const vp_upsample* ups, const vp_options* opt_in, void* stream)
{
    g_last_error.clear();
    if (!out) return fail(VP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (!ups || ups->n_types < 1 || !ups->types || ups->n_cells < 0 || (ups->n_cells > 0 && !ups->cell_type) ||
        !ups->f_start || !ups->src_start)
        return fail(VP_ERR_ARG, "incomplete upsampling description");
    if (ups->n_cells > (1LL << 30)) return fail(VP_ERR_ARG, "more than 2^30 cells");
    // types: host tables of [kind, n_q, n_p, qa, pa, qb, pb, 0] and concatenated matrices
    std::vector<int32_t> tinfo((size_t)ups->n_types * 8, 0);
    std::vector<int64_t> toff((size_t)ups->n_types * 2, 0);
    std::vector<double> mats;
    int32_t max_q = 1, max_p = 1, max_tmp = 1;
    for (int32_t t = 0; t < ups->n_types; ++t) {
        const vp_upsample_type& ty = ups->types[t];
        const std::string where = "upsampling type " + std::to_string(t) + ": ";
        if (ty.n_q < 1 || ty.n_p < 1 || ty.n_q > 1024 || ty.n_p > 1024)
            return fail(VP_ERR_ARG, where + "n_q and n_p must lie in [1, 1024]");
        int32_t* ti = tinfo.data() + 8 * (size_t)t;
        ti[1] = ty.n_q;
        ti[2] = ty.n_p;
        if (ty.kind == VP_UPS_TENSOR) {
            if (ty.qa < 1 || ty.pa < 1 || ty.qb < 1 || ty.pb < 1 || (int64_t)ty.qa * ty.qb != ty.n_q ||
                (int64_t)ty.pa * ty.pb != ty.n_p || (int64_t)ty.pa * ty.qb > 1024 || !ty.a || !ty.b)
                return fail(VP_ERR_ARG, where + "tensor factors do not match n_q, n_p (or pa*qb > 1024)");
            ti[0] = 1;
            ti[3] = ty.qa;
            ti[4] = ty.pa;
            ti[5] = ty.qb;
            ti[6] = ty.pb;
            toff[2 * (size_t)t] = (int64_t)mats.size();
            mats.insert(mats.end(), ty.a, ty.a + (size_t)ty.qa * ty.pa);
            toff[2 * (size_t)t + 1] = (int64_t)mats.size();
            mats.insert(mats.end(), ty.b, ty.b + (size_t)ty.qb * ty.pb);
            max_tmp = std::max(max_tmp, ty.pa * ty.qb);
        } else if (ty.kind == VP_UPS_DENSE) {
            if (!ty.mat) return fail(VP_ERR_ARG, where + "NULL matrix");
            toff[2 * (size_t)t] = (int64_t)mats.size();
            toff[2 * (size_t)t + 1] = (int64_t)mats.size();
            mats.insert(mats.end(), ty.mat, ty.mat + (size_t)ty.n_q * ty.n_p);
        } else {
            return fail(VP_ERR_ARG, where + "unknown kind");
        }
        max_q = std::max(max_q, ty.n_q);
        max_p = std::max(max_p, ty.n_p);
    }
    if (!finite_all(mats)) return fail(VP_ERR_ARG, "non-finite upsampling matrix");
    const int64_t nc = ups->n_cells;
    if (ups->f_start[0] != 0 || ups->src_start[0] != 0) return fail(VP_ERR_ARG, "cell ranges must start at 0");
    for (int64_t k = 0; k < nc; ++k) {
        const int32_t t = ups->cell_type[k];
        if (t < 0 || t >= ups->n_types) return fail(VP_ERR_ARG, "cell type out of range");
        if (ups->src_start[k + 1] - ups->src_start[k] != ups->types[t].n_q ||
            ups->f_start[k + 1] - ups->f_start[k] != ups->types[t].n_p)
            return fail(VP_ERR_ARG, "cell " + std::to_string(k) + ": node counts differ from its type");
    }
    if (ups->src_start[nc] != n_src) return fail(VP_ERR_ARG, "cells do not cover the n_src q-nodes");
    const int64_t n_f = ups->f_start[nc];
    if (n_f > (1LL << 30)) return fail(VP_ERR_ARG, "more than 2^30 density nodes");
    vp_options opt;
    int P, leaf, max_level, max_dens;
    vp_status st = plan_options(opt_in, opt, P, leaf, max_level, max_dens);
    if (st != VP_OK) return st;
    if (opt.kernel != VP_KERNEL_LAPLACE)
        return fail(VP_ERR_UNSUPPORTED, "the modified-Helmholtz kernel is available through vp_plan_create only");
    cudaStream_t s = (cudaStream_t)stream;
    ProblemIn in;
    st = copy_problem(in, n_src, src_xy, w, n_tgt, tgt_xy, corr_rowptr, corr_col, corr_val, nnz, s, n_f,
                      (opt.flags & VP_FLAG_FP64) != 0);
    if (st != VP_OK) return st;
    TreeOptions to;
    to.leaf = leaf;
    to.max_level = max_level;
    std::memcpy(to.root, opt.root, sizeof(to.root));
    Built B;
    std::string err = build_one(in, to, B, s);
    if (!err.empty()) return fail(VP_ERR_ARG, err);
    vp_plan p = new_plan(opt, P, leaf, max_dens);
    if (!p) return fail(VP_ERR_OOM, "host allocation");
    st = finalize(p, B, P, s);
    if (st == VP_OK) {
        std::vector<int32_t> ctype(ups->cell_type, ups->cell_type + nc);
        std::vector<int64_t> fst(ups->f_start, ups->f_start + nc + 1), sst(ups->src_start, ups->src_start + nc + 1);
        int32_t *d_ct = nullptr, *d_ti = nullptr;
        int64_t *d_fs = nullptr, *d_ss = nullptr, *d_to = nullptr;
        double* d_m = nullptr;
        cudaError_t e = p->upload(&d_ct, ctype, s);
        if (e == cudaSuccess) e = p->upload(&d_fs, fst, s);
        if (e == cudaSuccess) e = p->upload(&d_ss, sst, s);
        if (e == cudaSuccess) e = p->upload(&d_ti, tinfo, s);
        if (e == cudaSuccess) e = p->upload(&d_to, toff, s);
        if (e == cudaSuccess) e = p->upload(&d_m, mats, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "vp_plan_create_upsampled upload");
        } else {
            p->ups = true;
            DevUpsample& u = p->dups;
            u.n_cells = (int32_t)nc;
            u.n_types = ups->n_types;
            u.max_q = max_q;
            u.max_p = max_p;
            u.max_tmp = max_tmp;
            u.cell_type = d_ct;
            u.f_start = d_fs;
            u.src_start = d_ss;
            u.tinfo = d_ti;
            u.toff = d_to;
            u.mats = d_m;
        }
    }
    if (st != VP_OK) {
        delete p;
        return st;
    }
    *out = p;
    return VP_OK;
}

}  // extern "C"

extern "C" {

}  // extern "C"

namespace {

// Grouped correction product of one density chunk: out = A x (mode as in
// launch_out_grouped), x in caller order with leading dimension ld_x: exact
// fixed-point sums for float64 plans; float-float plans convert x to hi/lo
// floats first. Counts its launches.
vp_status grouped_apply(vp_plan p, int nd, const DevGroupedCSR& A, int64_t ncols, const int32_t* inv,
                        const double* w, const double* psi, const double* x, int64_t ld_x, double* out,
                        int64_t ld_out, int mode, int max_blocks, cudaStream_t s)
{
    if (p->arith == Arith::kF64) {
        VP_CUDA(launch_out_grouped64(nd, A, inv, w, psi, x, ld_x, out, ld_out, mode, max_blocks, s));
        p->last_launches += 1;
        return VP_OK;
    }
    VP_CUDA(launch_to_ff_rows(nd, (int32_t)ncols, x, ld_x, p->ws.xf, s));
    VP_CUDA(launch_out_grouped(nd, A, inv, w, psi, p->ws.xf, ncols, out, ld_out, mode, max_blocks, s));
    p->last_launches += 2;
    return VP_OK;
}

// Pi^T x of one density chunk from the forward grouped layout (modes as in
// launch_out_grouped; the columns are the density's points). Counts its launches.
vp_status adj_apply(vp_plan p, int nd, const int32_t* inv, const double* w, const double* psi, const double* x,
                    int64_t ld_x, double* out, int64_t ld_out, int mode, int max_blocks, cudaStream_t s)
{
    VP_CUDA(launch_adj_grouped(nd, p->gfwd, p->arith == Arith::kF64, x, ld_x, p->ws.adj_partial, inv, w, psi, out,
                               ld_out, mode, max_blocks, s));
    p->last_launches += 2;
    return VP_OK;
}

// The FMM of one density chunk for the plan's kernel (psi in tree order).
cudaError_t run_fmm(vp_plan p, int nd, const PassGeom& g, bool gradient, PhaseTimer* tm, cudaStream_t s)
{
    if (p->kernel == VP_KERNEL_MHELMHOLTZ)
        return launch_fmm_mhelm(p->P, p->dt, p->mh, p->tab.logtab, g, p->ws, !use_ff(p), tm, s);
    if (p->arith == Arith::kF64) return launch_fmm64(p->P, nd, p->dt, p->tab, g, p->ws, gradient, tm, s);
    return launch_fmm_potential(p->P, nd, p->dt, p->tab, g, p->ws, gradient, use_fp64(p), tm, s);
}

// The launch sequence of one evaluation, enqueued on s.
vp_status enqueue_eval(vp_plan p, int32_t ndens, const double* f, int64_t ld_f, double* out, int64_t ld_out,
                       cudaStream_t s)
{
    p->timer.stream = s;
    p->timer.used = 0;
    PassGeom g = forward_geom(p);
    p->last_launches = 0;
    for (int d0 = 0; d0 < ndens;) {
        const int nd = chunk_for(ndens - d0, p->nd_cap);
        // charges, P2M (+ M2M in the same launch on the float-float path, else per
        // level from level 2 up), M2L, L2L per level from level 3 down, leaf (+ slot
        // reduction), output
        // (the output launches are counted where they are made)
        if (p->kernel == VP_KERNEL_MHELMHOLTZ) {
            p->last_launches += 1 + mhelm_launches(p->dt.nlevels, p->dt.sym && use_ff(p));
        } else if (p->arith == Arith::kF64) {
            // charges, upward (P2M + M2M), M2L, L2L per level from 3, leaf (+ slot reduction)
            p->last_launches += 4 + (int64_t)std::max(0, p->dt.nlevels - 3) + (p->dt.sym ? 1 : 0);
        } else {
            const bool ffp = use_ff(p);
            p->last_launches += 4 + (ffp ? 0 : (int64_t)std::max(0, p->dt.nlevels - 3)) +
                                (int64_t)std::max(0, p->dt.nlevels - 3) + (p->dt.sym && ffp && nd <= 2 ? 1 : 0);
        }
        const double* fc = f + (int64_t)d0 * ld_f;
        double* oc = out + (int64_t)d0 * ld_out;
        // Pi f does not depend on the FMM: outside phase timing it runs beside the
        // FMM on the plan's low-priority stream, and the smooth part is added after
        const bool overlap = p->grouped && !p->timer.on && p->side_blocks > 0;
        if (overlap) {
            VP_CUDA(cudaEventRecord(p->ev_fork, s));
            VP_CUDA(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
            const vp_status st = grouped_apply(p, nd, p->gfwd, p->n_f, nullptr, nullptr, nullptr, fc, ld_f, oc,
                                               ld_out, kOutOverwrite, p->side_blocks, p->side);
            if (st != VP_OK) return st;
            VP_CUDA(cudaEventRecord(p->ev_join, p->side));
        }
        int id = p->timer.begin("charges");
        if (p->ups)
            VP_CUDA(launch_ups_charges(nd, p->dups, p->src_inv, p->w_sorted, fc, ld_f, p->ws.q, p->ws.qf, s));
        else
            VP_CUDA(launch_charges(nd, (int32_t)p->n_src, p->src_perm, p->w_sorted, fc, ld_f, p->ws.q, p->ws.qf, s));
        p->timer.end(id);
        VP_CUDA(run_fmm(p, nd, g, false, p->timer.on ? &p->timer : nullptr, s));
        id = p->timer.begin("out");
        if (overlap) {
            VP_CUDA(cudaStreamWaitEvent(s, p->ev_join, 0));
            VP_CUDA(launch_add_psi(nd, (int32_t)p->n_tgt, p->tgt_inv, nullptr, p->ws.psi, oc, ld_out, s));
            p->last_launches += 1;
        } else if (p->grouped) {
            const vp_status st = grouped_apply(p, nd, p->gfwd, p->n_f, p->tgt_inv, nullptr, p->ws.psi, fc, ld_f, oc,
                                               ld_out, kOutWithPsi, 0, s);
            if (st != VP_OK) return st;
        } else {
            VP_CUDA(launch_out_forward(nd, (int32_t)p->n_tgt, p->tgt_inv, p->ws.psi, p->rowptr, p->col, p->val, fc,
                                       ld_f, out + (int64_t)d0 * ld_out, ld_out, s));
            p->last_launches += 1;
        }
        p->timer.end(id);
        d0 += nd;
    }
    return VP_OK;
}

// Replays (or captures, then replays) the evaluation as a CUDA graph keyed by
// its arguments. Capture runs on a plan-owned stream in relaxed mode; the
// graph is launched on the caller's stream.
vp_status eval_graph(vp_plan p, int32_t ndens, const double* f, int64_t ld_f, double* out, int64_t ld_out,
                     cudaStream_t s)
{
    for (auto& gc : p->graphs)
        if (gc.f == f && gc.ld_f == ld_f && gc.out == out && gc.ld_out == ld_out && gc.ndens == ndens) {
            p->last_launches = gc.launches;
            VP_CUDA(cudaGraphLaunch(gc.exec, s));
            return VP_OK;
        }
    if (!p->cap_stream) {
        // captured FMM kernels take precedence over the correction product beside them
        int least = 0, greatest = 0;
        VP_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        VP_CUDA(cudaStreamCreateWithPriority(&p->cap_stream, cudaStreamNonBlocking, greatest));
    }
    // order the capture after the caller's pending work on s, and the replay after the capture
    VP_CUDA(cudaStreamSynchronize(s));
    VP_CUDA(cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed));
    vp_status st = enqueue_eval(p, ndens, f, ld_f, out, ld_out, p->cap_stream);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(p->cap_stream, &graph);
    if (st != VP_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    if (p->graphs.size() >= 8) {
        cudaGraphExecDestroy(p->graphs.front().exec);
        p->graphs.erase(p->graphs.begin());
    }
    p->graphs.push_back(vp_plan_s::GraphEntry{f, ld_f, out, ld_out, ndens, p->last_launches, exec});
    VP_CUDA(cudaGraphLaunch(exec, s));
    return VP_OK;
}

}  // namespace

extern "C" {

vp_status vp_eval(vp_plan p, int32_t ndens, const double* f, int64_t ld_f, double* out, int64_t ld_out,
                  void* stream)
{
    vp_status st = check_plan(p);
    if (st != VP_OK) return st;
    if (ndens < 0) return fail(VP_ERR_ARG, "ndens < 0");
    if (ndens == 0 || p->n_tgt == 0) return VP_OK;
    if (!out || (p->n_f > 0 && !f)) return fail(VP_ERR_ARG, "NULL density or output");
    if (ld_f < p->n_f || ld_out < p->n_tgt) return fail(VP_ERR_ARG, "leading dimension too small");
    cudaStream_t s = (cudaStream_t)stream;
    if ((p->flags & VP_FLAG_GRAPH) && !p->timer.on) return eval_graph(p, ndens, f, ld_f, out, ld_out, s);
    return enqueue_eval(p, ndens, f, ld_f, out, ld_out, s);
}

vp_status vp_eval_adjoint(vp_plan p, int32_t ndens, const double* g, int64_t ld_g, double* grad_f, int64_t ld_gf,
                          const double* f, int64_t ld_f, double* grad_tgt, void* stream)
{
    vp_status st = check_plan(p);
    if (st != VP_OK) return st;
    if (ndens < 0) return fail(VP_ERR_ARG, "ndens < 0");
    cudaStream_t s = (cudaStream_t)stream;
    if (grad_tgt && p->n_tgt > 0) {
        if (ndens == 0) {
            VP_CUDA(cudaMemsetAsync(grad_tgt, 0, sizeof(double) * 2 * p->n_tgt, s));
        } else if (!g || (p->n_f > 0 && !f) || ld_g < p->n_tgt || ld_f < p->n_f) {
            return fail(VP_ERR_ARG, "target gradient needs g and f with valid leading dimensions");
        }
    }
    if (grad_f && p->n_f > 0) {
        if (ndens == 0) return VP_OK;
        if ((p->n_tgt > 0 && !g) || ld_g < p->n_tgt || ld_gf < p->n_f)
            return fail(VP_ERR_ARG, "grad_f needs g with valid leading dimensions");
    }
    if (grad_tgt && p->kernel != VP_KERNEL_LAPLACE)
        return fail(VP_ERR_UNSUPPORTED, "target gradients are available for the Laplace kernel only");
    if (ndens == 0) return VP_OK;
    p->timer.stream = s;
    p->timer.used = 0;
    const int64_t fwd_launches = p->last_launches;  // the stats report the last vp_eval
    if (grad_f && p->n_f > 0) {
        PassGeom gg = adjoint_geom(p);
        for (int d0 = 0; d0 < ndens;) {
            const int nd = chunk_for(ndens - d0, p->nd_cap);
            const double* gc = g + (int64_t)d0 * ld_g;
            double* gfc0 = grad_f + (int64_t)d0 * ld_gf;
            // Pi^T g beside the transposed FMM (as in the forward evaluation)
            const bool overlap = p->grouped && !p->ups && p->side_blocks > 0;
            if (overlap) {
                VP_CUDA(cudaEventRecord(p->ev_fork, s));
                VP_CUDA(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
                const vp_status st = adj_apply(p, nd, nullptr, nullptr, nullptr, gc, ld_g,
                                                   gfc0, ld_gf, kOutOverwrite, p->side_blocks, p->side);
                if (st != VP_OK) return st;
                VP_CUDA(cudaEventRecord(p->ev_join, p->side));
            }
            VP_CUDA(launch_charges(nd, (int32_t)p->n_tgt, p->tgt_perm, nullptr, gc, ld_g, p->ws.q, p->ws.qf, s));
            VP_CUDA(run_fmm(p, nd, gg, false, nullptr, s));
            if (overlap) {
                VP_CUDA(cudaStreamWaitEvent(s, p->ev_join, 0));
                VP_CUDA(launch_add_psi(nd, (int32_t)p->n_f, p->src_inv, p->w_sorted, p->ws.psi, gfc0, ld_gf, s));
            } else if (p->ups) {
                // grad_f = O^T (w * transposed sum at the q-nodes), then += Pi^T g
                double* gfc = grad_f + (int64_t)d0 * ld_gf;
                VP_CUDA(launch_ups_adjoint(nd, p->dups, p->src_inv, p->w_sorted, p->ws.psi, gfc, ld_gf, s));
                if (p->grouped) {
                    const vp_status st = adj_apply(p, nd, nullptr, nullptr, nullptr, gc, ld_g,
                                                       gfc, ld_gf, kOutAccumulate, 0, s);
                    if (st != VP_OK) return st;
                } else if (p->cptr) {
                    VP_CUDA(launch_out_adjoint(nd, (int32_t)p->n_f, nullptr, nullptr, nullptr, p->cptr, p->crow,
                                               p->cval, gc, ld_g, gfc, ld_gf, s));
                }
            } else if (p->grouped) {
                const vp_status st = adj_apply(p, nd, p->src_inv, p->w_sorted, p->ws.psi, gc,
                                                   ld_g, grad_f + (int64_t)d0 * ld_gf, ld_gf, kOutWithPsi, 0, s);
                if (st != VP_OK) return st;
            } else {
                VP_CUDA(launch_out_adjoint(nd, (int32_t)p->n_src, p->src_inv, p->w_sorted, p->ws.psi, p->cptr,
                                           p->crow, p->cval, gc, ld_g, grad_f + (int64_t)d0 * ld_gf, ld_gf, s));
            }
            d0 += nd;
        }
    }
    if (grad_tgt && p->n_tgt > 0) {
        PassGeom gf = forward_geom(p);
        for (int d0 = 0; d0 < ndens;) {
            const int nd = chunk_for(ndens - d0, p->nd_cap);
            const double* fc = f + (int64_t)d0 * ld_f;
            if (p->ups)
                VP_CUDA(launch_ups_charges(nd, p->dups, p->src_inv, p->w_sorted, fc, ld_f, p->ws.q, p->ws.qf, s));
            else
                VP_CUDA(launch_charges(nd, (int32_t)p->n_src, p->src_perm, p->w_sorted, fc, ld_f, p->ws.q, p->ws.qf,
                                       s));
            VP_CUDA(run_fmm(p, nd, gf, true, nullptr, s));
            VP_CUDA(launch_grad_out(nd, d0 > 0, (int32_t)p->n_tgt, p->tgt_perm, p->ws.psi, g + (int64_t)d0 * ld_g,
                                    ld_g, grad_tgt, s));
            d0 += nd;
        }
    }
    p->last_launches = fwd_launches;
    return VP_OK;
}

vp_status vp_eval_batch(int32_t nplans, const vp_plan* plans, const int32_t* ndens, const double* const* f,
                        const int64_t* ld_f, double* const* out, const int64_t* ld_out, void* stream)
{
    if (nplans < 0) return fail(VP_ERR_ARG, "nplans < 0");
    if (nplans == 0) return VP_OK;
    if (!plans || !ndens || !f || !ld_f || !out || !ld_out) return fail(VP_ERR_ARG, "NULL batch array");
    for (int32_t k = 0; k < nplans; ++k) {
        const vp_status st = vp_eval(plans[k], ndens[k], f[k], ld_f[k], out[k], ld_out[k], stream);
        if (st != VP_OK) return st;
    }
    return VP_OK;
}

vp_status vp_eval_host(vp_plan p, int32_t ndens, const double* f_host, double* out_host, void* stream)
{
    vp_status st = check_plan(p);
    if (st != VP_OK) return st;
    if (ndens < 0) return fail(VP_ERR_ARG, "ndens < 0");
    if (ndens == 0) return VP_OK;
    if ((p->n_f > 0 && !f_host) || (p->n_tgt > 0 && !out_host)) return fail(VP_ERR_ARG, "NULL host buffer");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t nf = (size_t)ndens * (size_t)p->n_f, no = (size_t)ndens * (size_t)p->n_tgt;
    if (nf + no > p->stage_cap) {
        if (p->stage) cudaFree(p->stage);
        p->stage = nullptr;
        p->stage_cap = 0;
        void* q = nullptr;
        VP_CUDA(cudaMalloc(&q, (nf + no) * sizeof(double)));
        p->stage = (double*)q;
        p->stage_cap = nf + no;
    }
    double* df = p->stage;
    double* dout = p->stage + nf;
    if (nf) VP_CUDA(cudaMemcpyAsync(df, f_host, nf * sizeof(double), cudaMemcpyHostToDevice, s));
    st = vp_eval(p, ndens, df, p->n_f, dout, p->n_tgt, stream);
    if (st != VP_OK) return st;
    if (no) VP_CUDA(cudaMemcpyAsync(out_host, dout, no * sizeof(double), cudaMemcpyDeviceToHost, s));
    VP_CUDA(cudaStreamSynchronize(s));
    return VP_OK;
}

vp_status vp_plan_info(vp_plan p, vp_plan_stats* o)
{
    if (!p || !p->alive) return fail(VP_ERR_STATE, "invalid plan");
    if (!o) return fail(VP_ERR_ARG, "NULL stats");
    std::memset(o, 0, sizeof(*o));
    o->n_src = p->n_src;
    o->n_tgt = p->n_tgt;
    o->nnz = p->nnz;
    o->p_fmm = p->P;
    o->leaf = p->leaf;
    o->max_dens = p->max_dens;
    o->n_levels = p->stat_levels;
    o->n_boxes = p->stat_boxes;
    o->n_leaves = p->stat_leaves;
    o->n_u_pairs = p->stat_u;
    o->n_v_pairs = p->stat_v;
    o->n_w_pairs = p->stat_w;
    o->n_x_pairs = p->stat_x;
    o->p2p_pairs = p->p2p_pairs;
    o->last_launches = p->last_launches;
    o->n_problems = p->n_problems;
    o->root[0] = p->stat_root[0];
    o->root[1] = p->stat_root[1];
    o->root[2] = p->stat_root[2];
    o->n_f = p->n_f;
    o->n_cells = p->ups ? p->dups.n_cells : 0;
    o->sym_slots = p->dt.sym ? p->dt.sym_slots : 0;
    o->p2p_evals = p->dt.sym ? p->p2p_evals : p->p2p_pairs;
    o->kernel = p->kernel;
    o->near_terms = p->kernel == VP_KERNEL_MHELMHOLTZ ? p->mh.near_deg + 1 : 0;
    o->lambda = p->kernel == VP_KERNEL_MHELMHOLTZ ? p->mh.lambda : 0.0;
    o->near_ops = p->kernel == VP_KERNEL_MHELMHOLTZ ? p->mh_near_ops : 0;
    return VP_OK;
}

vp_status vp_plan_phase_times(vp_plan p, int32_t cap, const char** names, double* ms, int32_t* n)
{
    if (!p || !p->alive) return fail(VP_ERR_STATE, "invalid plan");
    if (!n) return fail(VP_ERR_ARG, "NULL count");
    const PhaseTimer& t = p->timer;
    *n = (int32_t)t.names.size();
    if (!t.on) {
        *n = 0;
        return VP_OK;
    }
    std::vector<double> sum(t.names.size(), 0.0);
    for (int i = 0; i < t.used; ++i) {
        VP_CUDA(cudaEventSynchronize(t.pool[2 * i + 1]));
        float x = 0.f;
        VP_CUDA(cudaEventElapsedTime(&x, t.pool[2 * i], t.pool[2 * i + 1]));
        sum[(size_t)t.phase_of[(size_t)i]] += x;
    }
    for (int32_t i = 0; i < *n && i < cap; ++i) {
        if (names) names[i] = t.names[(size_t)i].c_str();
        if (ms) ms[i] = sum[(size_t)i];
    }
    return VP_OK;
}

vp_status vp_plan_set_flags(vp_plan p, uint32_t flags)
{
    if (!p || !p->alive) return fail(VP_ERR_STATE, "invalid plan");
    const uint32_t runtime = VP_FLAG_TIMING | VP_FLAG_GRAPH;
    if ((flags & ~runtime) != (p->flags & ~runtime))
        return fail(VP_ERR_ARG, "only VP_FLAG_TIMING and VP_FLAG_GRAPH can change after plan creation");
    p->flags = flags;
    p->timer.on = (flags & VP_FLAG_TIMING) != 0;
    return VP_OK;
}

vp_status vp_plan_set_overlap(vp_plan p, int32_t blocks_per_sm)
{
    vp_status st = check_plan(p);
    if (st != VP_OK) return st;
    if (blocks_per_sm < 0 || blocks_per_sm > 64) return fail(VP_ERR_ARG, "blocks_per_sm outside 0..64");
    p->side_blocks = p->side ? blocks_per_sm * p->sms : 0;
    for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);  // captured with the old schedule
    p->graphs.clear();
    return VP_OK;
}

vp_status vp_green_eval_host(int32_t kernel, double lambda, int64_t n, const double* r, double* g)
{
    if (n < 0 || (n > 0 && (!r || !g))) return fail(VP_ERR_ARG, "NULL pointer or n < 0");
    if (kernel != VP_KERNEL_LAPLACE && kernel != VP_KERNEL_MHELMHOLTZ) return fail(VP_ERR_ARG, "unknown kernel");
    if (kernel == VP_KERNEL_MHELMHOLTZ && !(lambda > 0.0 && std::isfinite(lambda)))
        return fail(VP_ERR_ARG, "the modified-Helmholtz kernel needs a finite lambda > 0");
    for (int64_t i = 0; i < n; ++i)
        if (!(r[i] > 0.0)) return fail(VP_ERR_ARG, "distances must be > 0");
    for (int64_t i = 0; i < n; ++i)
        g[i] = kernel == VP_KERNEL_LAPLACE ? -0.159154943091895335768883763372514362 * std::log(r[i])
                                           : green_mhelm_host(lambda, r[i]);
    return VP_OK;
}

vp_status vp_plan_destroy(vp_plan p)
{
    if (!p) return VP_OK;
    if (!p->alive) return fail(VP_ERR_STATE, "plan destroyed twice");
    p->alive = false;
    delete p;
    return VP_OK;
}

// ---------------------------------------------------------------------------
struct vp_tree_s {
    Tree t;
};

vp_status vp_tree_build(vp_tree* out, int64_t n_src, const double* src_xy, int64_t n_tgt, const double* tgt_xy,
                        const vp_options* opt_in)
{
    if (!out) return fail(VP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_src < 0 || n_tgt < 0) return fail(VP_ERR_ARG, "negative size");
    if ((n_src > 0 && !src_xy) || (n_tgt > 0 && !tgt_xy)) return fail(VP_ERR_ARG, "NULL point array");
    vp_options opt;
    std::memset(&opt, 0, sizeof(opt));
    if (opt_in) opt = *opt_in;
    TreeOptions to;
    to.leaf = opt.leaf == 0 ? 64 : opt.leaf;
    to.max_level = opt.max_level == 0 ? 24 : opt.max_level;
    to.root[0] = opt.root[0];
    to.root[1] = opt.root[1];
    to.root[2] = opt.root[2];
    vp_tree t = new (std::nothrow) vp_tree_s();
    if (!t) return fail(VP_ERR_OOM, "host allocation");
    std::string err = build_tree(n_src, src_xy, n_tgt, tgt_xy, to, t->t);
    if (!err.empty()) {
        delete t;
        return fail(VP_ERR_ARG, err);
    }
    *out = t;
    return VP_OK;
}

vp_status vp_tree_build_device(vp_tree* out, int64_t n_src, const double* src_xy, int64_t n_tgt,
                               const double* tgt_xy, const vp_options* opt_in, void* stream)
{
    if (!out) return fail(VP_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (n_src < 0 || n_tgt < 0) return fail(VP_ERR_ARG, "negative size");
    if ((n_src > 0 && !src_xy) || (n_tgt > 0 && !tgt_xy)) return fail(VP_ERR_ARG, "NULL point array");
    vp_options opt;
    std::memset(&opt, 0, sizeof(opt));
    if (opt_in) opt = *opt_in;
    TreeOptions to;
    to.leaf = opt.leaf == 0 ? 64 : opt.leaf;
    to.max_level = opt.max_level == 0 ? 24 : opt.max_level;
    to.root[0] = opt.root[0];
    to.root[1] = opt.root[1];
    to.root[2] = opt.root[2];
    vp_tree t = new (std::nothrow) vp_tree_s();
    if (!t) return fail(VP_ERR_OOM, "host allocation");
    std::string err = build_tree_gpu(n_src, src_xy, n_tgt, tgt_xy, to, t->t, (cudaStream_t)stream);
    if (!err.empty()) {
        delete t;
        return fail(err.rfind("CUDA:", 0) == 0 ? VP_ERR_CUDA : VP_ERR_ARG, err);
    }
    *out = t;
    return VP_OK;
}

vp_status vp_tree_get(vp_tree tree, int32_t which, int32_t* dst, int64_t* count)
{
    if (!tree || !count) return fail(VP_ERR_ARG, "NULL tree or count");
    const Tree& T = tree->t;
    std::vector<int32_t> tmp;
    const std::vector<int32_t>* src = nullptr;
    auto pairs = [&](const std::vector<int32_t>& a, const std::vector<int32_t>& b) {
        tmp.resize(a.size() * 2);
        for (size_t i = 0; i < a.size(); ++i) {
            tmp[2 * i] = a[i];
            tmp[2 * i + 1] = b[i];
        }
        src = &tmp;
    };
    switch (which) {
        case VP_TREE_BOX_LEVEL: src = &T.level; break;
        case VP_TREE_BOX_IXY: pairs(T.ix, T.iy); break;
        case VP_TREE_BOX_PARENT: src = &T.parent; break;
        case VP_TREE_BOX_LEAF: src = &T.is_leaf; break;
        case VP_TREE_BOX_SRC: pairs(T.src_begin, T.src_end); break;
        case VP_TREE_BOX_TGT: pairs(T.tgt_begin, T.tgt_end); break;
        case VP_TREE_SRC_PERM: src = &T.src_perm; break;
        case VP_TREE_TGT_PERM: src = &T.tgt_perm; break;
        case VP_TREE_U_PTR: src = &T.u_ptr; break;
        case VP_TREE_U_IDX: src = &T.u_idx; break;
        case VP_TREE_V_PTR: src = &T.v_ptr; break;
        case VP_TREE_V_IDX: src = &T.v_idx; break;
        case VP_TREE_W_PTR: src = &T.w_ptr; break;
        case VP_TREE_W_IDX: src = &T.w_idx; break;
        case VP_TREE_X_PTR: src = &T.x_ptr; break;
        case VP_TREE_X_IDX: src = &T.x_idx; break;
        default: return fail(VP_ERR_ARG, "unknown tree array");
    }
    *count = (int64_t)src->size();
    if (dst && !src->empty()) std::memcpy(dst, src->data(), src->size() * sizeof(int32_t));
    return VP_OK;
}

vp_status vp_tree_destroy(vp_tree tree)
{
    delete tree;
    return VP_OK;
}

}  // extern "C"
