// api.cu -- the C ABI of include/nnqs.h: argument validation, host-side
// lattice and symmetry tables (Sec. 2.1 Eq. 1, Sec. 3.1 Eqs. 4-6), device
// memory of the model, and dispatch to the kernels.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/nnqs.h"
#include "common.cuh"
#include "kernels.h"

using namespace nnqs;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *where)
{
    return fail(e == cudaErrorMemoryAllocation ? NNQS_ENOMEM : NNQS_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define NNQS_CUDA(call)                                 \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

// ---------------------------------------------------------------------------
// Lattice tables
// ---------------------------------------------------------------------------
int site(int L, int x, int y) { return ((x % L + L) % L) + L * ((y % L + L) % L); }

// J1 (+x), J1 (+y), J2 (+x+y), J2 (+x-y) for each site in increasing index
void make_bonds(int L, std::vector<int16_t> &bi, std::vector<int16_t> &bj, std::vector<uint8_t> &bt)
{
    const int dx[4] = {1, 0, 1, 1}, dy[4] = {0, 1, 1, -1};
    for (int i = 0; i < L * L; ++i)
        for (int d = 0; d < 4; ++d) {
            bi.push_back((int16_t)i);
            bj.push_back((int16_t)site(L, i % L + dx[d], i / L + dy[d]));
            bt.push_back(d < 2 ? 1 : 2);
        }
}

// C4v element l acting on (x, y) about site 0: E, C4, C2, C4^3, x-mirror,
// y-mirror, diagonal mirror, anti-diagonal mirror, as 2x2 integer matrices.
const int kPoint[8][4] = {{1, 0, 0, 1},  {0, -1, 1, 0}, {-1, 0, 0, -1}, {0, 1, -1, 0},
                          {-1, 0, 0, 1}, {1, 0, 0, -1}, {0, 1, 1, 0},   {0, -1, -1, 0}};
// one-dimensional irreps (A1, A2, B1, B2) on the classes {E}, {C4, C4^3}, {C2},
// {axis mirrors}, {diagonal mirrors}
int c4v_character(int irrep, int l)
{
    const int rot = (l == 1 || l == 3) ? 1 : 0, axis = (l == 4 || l == 5), diag = (l == 6 || l == 7);
    const int c4_sign = (irrep >= 2) ? -1 : 1;                 // B irreps are odd under C4
    const int axis_sign = (irrep == 1 || irrep == 3) ? -1 : 1;  // A2, B2 odd under axis mirrors
    int c = 1;
    if (rot) c = c4_sign;
    if (axis) c = axis_sign;
    if (diag) c = c4_sign * axis_sign;  // sigma_d = C4 * sigma_axis
    return c;
}

int make_group(const nnqs_desc &d, std::vector<uint8_t> &perm, std::vector<double> &chi)
{
    const int L = d.L, N = L * L;
    std::vector<int> ops;
    if (!d.project_point_group) ops = {0};
    else if (d.momentum == NNQS_K00 || d.momentum == NNQS_KPIPI) ops = {0, 1, 2, 3, 4, 5, 6, 7};
    else ops = {0, 2, 4, 5};  // little group of (pi,0) / (0,pi)
    const int nt = d.project_translations ? N : 1;
    int G = 0;
    for (int l : ops)
        for (int t = 0; t < nt; ++t) {
            const int m = t % L, n = t / L;
            int ph = 1;
            if (d.momentum == NNQS_KPIPI && ((m + n) & 1)) ph = -1;
            if (d.momentum == NNQS_KPI0 && (m & 1)) ph = -1;
            if (d.momentum == NNQS_K0PI && (n & 1)) ph = -1;
            chi.push_back((double)(ph * c4v_character(d.irrep, l)));
            const int *R = kPoint[l];
            for (int i = 0; i < N; ++i) {
                const int x = i % L, y = i / L;
                perm.push_back((uint8_t)site(L, R[0] * x + R[1] * y + m, R[2] * x + R[3] * y + n));
            }
            ++G;
        }
    return G;
}

}  // namespace

// ---------------------------------------------------------------------------
// Model
// ---------------------------------------------------------------------------
struct nnqs_model {
    nnqs_desc d;
    int N, G, nsign, nwords, nbonds, nsm, device;
    int Mp;  // row stride of the connected-configuration tables
    int64_t P;
    bool fp64;
    bool can_vanish;  // some group element carries character -1: amplitudes can vanish by symmetry
    uint8_t *perm = nullptr;
    int16_t *bi = nullptr, *bj = nullptr;
    uint8_t *bt = nullptr;
    void *chi = nullptr;
    double *params = nullptr;
    void *Wt = nullptr, *b = nullptr, *a = nullptr, *logc = nullptr, *X = nullptr, *XA = nullptr;
    void *Tb = nullptr, *Cb = nullptr, *S4 = nullptr, *CS = nullptr, *ES = nullptr;
    uint16_t *bperm = nullptr;
    // tensor-core path (NNQS_BF16X2 / NNQS_BF16X3)
    int ns = 0;                  // bf16 terms of the split (0: tensor-core path off)
    uint16_t *bimg = nullptr;    // shared-memory images of the split weights
    uint16_t *pinv = nullptr;    // inverse permutations [G][round16(N)]
    int *status = nullptr;
    unsigned long long *chk = nullptr;  // checked mode: first configuration outside Sz = 0
    void *eft = nullptr;                // FP32 E_loc: paired per-bond tables (nullptr: not supported)
    void *lft = nullptr;                // FP32 h1/h2: paired per-site factors (nullptr: not supported)
    void *ws = nullptr;
    size_t ws_bytes = 0;
};

namespace {

template <typename T> DevModel<T> view(const nnqs_model *m)
{
    DevModel<T> v;
    v.L = m->d.L; v.N = m->N; v.K = m->d.K; v.M = m->d.M; v.G = m->G; v.nsign = m->nsign;
    v.Mp = m->Mp;
    v.use_bias = m->d.use_bias; v.nbonds = m->nbonds; v.nwords = m->nwords; v.chiP = m->d.spin_inversion;
    v.J1 = (T)m->d.J1; v.J2 = (T)m->d.J2;
    v.perm = m->perm; v.chi = (const T *)m->chi;
    v.Wt = (const cx<T> *)m->Wt; v.bvec = (const cx<T> *)m->b; v.avec = (const cx<T> *)m->a;
    v.logc = (const cx<T> *)m->logc; v.X = (const cx2<T> *)m->X; v.XA = (const cx2<T> *)m->XA;
    v.bond_i = m->bi; v.bond_j = m->bj; v.bond_t = m->bt;
    v.Tb = (const cx<T> *)m->Tb; v.Cb = (const cx<T> *)m->Cb; v.S4 = (const cx<T> *)m->S4; v.CS = (const cx<T> *)m->CS;
    v.bperm = m->bperm;
    v.ES = (const sc<T> *)m->ES;
    v.status = m->status;
    return v;
}

// Test hook: NNQS_TEST_ELOC_ENGINE=old runs E_loc on the general connected-
// configuration engine even where the shared-memory form applies (for
// comparisons of the two).  Unset in normal use.
bool test_old_engine()
{
    const char *v = getenv("NNQS_TEST_ELOC_ENGINE");
    return v && v[0] == 'o';
}

// Test hook: NNQS_TEST_WORKSPACE_CAP=<bytes> makes every workspace growth
// beyond that size fail as a refused allocation (NNQS_ENOMEM).  Unset in
// normal use.
size_t workspace_cap()
{
    const char *v = getenv("NNQS_TEST_WORKSPACE_CAP");
    if (!v || !*v) return (size_t)-1;
    char *end = nullptr;
    const unsigned long long c = strtoull(v, &end, 10);
    return (end && *end == 0) ? (size_t)c : (size_t)-1;
}

int ensure_ws(nnqs_model *m, size_t bytes)
{
    if (bytes <= m->ws_bytes) return NNQS_OK;
    if (bytes > workspace_cap())
        return fail(NNQS_ENOMEM, "workspace of %zu bytes refused (test cap %zu)", bytes, workspace_cap());
    if (m->ws) {
        cudaDeviceSynchronize();
        cudaFree(m->ws);
        m->ws = nullptr;
        m->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&m->ws, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NNQS_ENOMEM, "workspace of %zu bytes refused: %s", bytes, cudaGetErrorString(e));
    }
    m->ws_bytes = bytes;
    return NNQS_OK;
}

int check_model(const nnqs_model *m)
{
    if (!m) return fail(NNQS_EINVAL, "model is NULL");
    return NNQS_OK;
}

template <typename F> int with_device(const nnqs_model *m, F &&f)
{
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != m->device) cudaSetDevice(m->device);
    const int rc = f();
    if (cur != m->device && cur >= 0) cudaSetDevice(cur);
    return rc;
}

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Post-pass for configurations annihilated by the projection (models with a
// character -1 only): log psi = -inf (mode 0); E_loc / h1 / h2 = NaN and
// NNQS_ERANGE in the status word (mode 1).
cudaError_t mark_vanishing(const nnqs_model *m, const uint64_t *cfg, int64_t n, int mode, double *o1, double *o2,
                           cudaStream_t st);

// h1 and h2 of n configurations on the model's engine: the shared-memory
// site-table form where it applies (FP32), else the general one.
cudaError_t lanczos_h(const nnqs_model *m, const uint64_t *cfg, int64_t n, double *h1, double *h2, cudaStream_t st);

// Checked mode (desc.check_inputs): rejects a batch of configurations with
// NNQS_EINVAL if any lies outside the Sz = 0 sector or sets bits past site
// N - 1.  Runs one small kernel and synchronises the stream; a no-op when the
// mode is off.  Called with the model's device current.
int check_cfg(const nnqs_model *m, const uint64_t *cfg, int64_t n, cudaStream_t st)
{
    if (!m->d.check_inputs || n <= 0) return NNQS_OK;
    cudaError_t e = launch_check_sz0(cfg, n, m->nwords, m->N, m->chk, st);
    unsigned long long bad = ~0ull;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, m->chk, sizeof bad, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "input check");
    if (bad == ~0ull) return NNQS_OK;
    uint64_t w[kMaxWords] = {};
    e = cudaMemcpy(w, cfg + (size_t)bad * m->nwords, (size_t)m->nwords * sizeof(uint64_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "input check");
    int up = 0;
    for (int k = 0; k < m->nwords; ++k) up += __builtin_popcountll(w[k]);
    return fail(NNQS_EINVAL, "configuration %llu is not a valid Sz = 0 state of %d sites (%d bits set)", bad, m->N,
                up);
}

cudaError_t lanczos_h(const nnqs_model *m, const uint64_t *cfg, int64_t n, double *h1, double *h2, cudaStream_t st)
{
    if (m->fp64) return launch_ratio(view<double>(m), cfg, n, 1, h1, h2, m->nsm, st);
    if (m->lft && !test_old_engine()) return launch_lanczos_fast(view<float>(m), m->lft, cfg, n, h1, h2, m->nsm, st);
    return launch_ratio(view<float>(m), cfg, n, 1, h1, h2, m->nsm, st);
}

cudaError_t mark_vanishing(const nnqs_model *m, const uint64_t *cfg, int64_t n, int mode, double *o1, double *o2,
                           cudaStream_t st)
{
    if (!m->can_vanish || n <= 0) return cudaSuccess;
    return m->fp64 ? launch_mark_vanishing(view<double>(m), cfg, n, mode, o1, o2, st)
                   : launch_mark_vanishing(view<float>(m), cfg, n, mode, o1, o2, st);
}

}  // namespace

extern "C" {

const char *nnqs_last_error(void) { return g_err.c_str(); }

// mp_min: smallest row stride of the connected-configuration tables (0: the
// narrowest that the model's width allows)
static int create_model(const nnqs_desc *desc, int mp_min, nnqs_model **out)
{
    if (!desc || !out) return fail(NNQS_EINVAL, "desc and out must be non-NULL");
    *out = nullptr;
    const nnqs_desc d = *desc;
    if (d.L < 4 || (d.L & 1)) return fail(NNQS_EUNSUPPORTED, "L must be even and >= 4 (got %d)", d.L);
    if (d.L > kMaxL) return fail(NNQS_EUNSUPPORTED, "L > %d is not supported", kMaxL);
    if (d.K < 1 || d.K > kMaxK) return fail(NNQS_EUNSUPPORTED, "K must be in 1..%d", kMaxK);
    if (d.M < 1 || d.M > kMaxM) return fail(NNQS_EUNSUPPORTED, "M must be in 1..%d", kMaxM);
    if (d.momentum < 0 || d.momentum > 3) return fail(NNQS_EINVAL, "momentum must be 0..3");
    if (d.irrep < 0 || d.irrep > 3) return fail(NNQS_EINVAL, "irrep must be 0..3");
    if (d.spin_inversion < -1 || d.spin_inversion > 1) return fail(NNQS_EINVAL, "spin_inversion must be -1, 0 or 1");
    if (!d.use_bias && d.spin_inversion == -1)
        return fail(NNQS_EINVAL, "spin_inversion = -1 without biases: the projection vanishes identically");
    if (d.precision < NNQS_FP64 || d.precision > NNQS_BF16X3) return fail(NNQS_EINVAL, "unknown precision %d", d.precision);
    if (!(d.J1 == d.J1) || !(d.J2 == d.J2)) return fail(NNQS_EINVAL, "J1, J2 must be finite");

    nnqs_model *m = new nnqs_model();
    m->d = d;
    m->N = d.L * d.L;
    m->nwords = (m->N + 63) / 64;
    m->nsign = d.spin_inversion ? 2 : 1;
    m->P = (int64_t)d.K * (1 + m->N + d.M + (int64_t)d.M * m->N);
    m->fp64 = d.precision == NNQS_FP64;
    m->Mp = conn_mpad(d.M) > mp_min ? conn_mpad(d.M) : mp_min;
    cudaGetDevice(&m->device);
    cudaDeviceGetAttribute(&m->nsm, cudaDevAttrMultiProcessorCount, m->device);

    std::vector<int16_t> bi, bj;
    std::vector<uint8_t> bt, perm;
    std::vector<double> chi;
    make_bonds(d.L, bi, bj, bt);
    m->nbonds = (int)bi.size();
    m->G = make_group(d, perm, chi);
    {
        const int inv_char = d.spin_inversion ? d.spin_inversion : (d.use_bias ? 0 : 1);
        m->can_vanish = inv_char < 0;
        for (double c : chi) m->can_vanish = m->can_vanish || c < 0;
    }

    auto cleanup = [&](int rc) { nnqs_destroy(m); return rc; };
    const size_t ts = m->fp64 ? sizeof(double) : sizeof(float);
    const size_t K = d.K, M = d.M, N = m->N;
#define ALLOC(ptr, bytes)                                                        \
    do {                                                                         \
        cudaError_t e_ = cudaMalloc((void **)&(ptr), (bytes));                   \
        if (e_ != cudaSuccess) { cudaGetLastError(); return cleanup(cuda_fail(e_, "cudaMalloc")); } \
    } while (0)
    ALLOC(m->perm, perm.size());
    ALLOC(m->bi, bi.size() * 2);
    ALLOC(m->bj, bj.size() * 2);
    ALLOC(m->bt, bt.size());
    ALLOC(m->chi, chi.size() * ts);
    ALLOC(m->params, (size_t)m->P * 2 * sizeof(double));
    ALLOC(m->Wt, K * N * M * 2 * ts);
    ALLOC(m->b, K * M * 2 * ts);
    ALLOC(m->a, K * N * 2 * ts);
    ALLOC(m->logc, K * 2 * ts);
    ALLOC(m->X, K * N * M * 4 * ts);
    ALLOC(m->XA, K * N * 4 * ts);
    const size_t Mp = (size_t)m->Mp;
    ALLOC(m->Tb, K * 2 * bi.size() * Mp * 2 * ts);
    ALLOC(m->Cb, K * bi.size() * 2 * ts);
    ALLOC(m->S4, K * 2 * N * Mp * 2 * ts);
    ALLOC(m->CS, K * N * 2 * ts);
    ALLOC(m->ES, K * 2 * N * (m->fp64 ? sizeof(sc<double>) : sizeof(sc<float>)));
    ALLOC(m->bperm, (size_t)m->G * bi.size() * sizeof(uint16_t));
    ALLOC(m->status, sizeof(int));
    ALLOC(m->chk, sizeof(unsigned long long));
    if (!m->fp64) {
        DevModel<float> v{};
        v.K = d.K; v.M = d.M; v.N = m->N; v.G = m->G; v.nbonds = (int)bi.size(); v.Mp = m->Mp;
        if (eloc_fast_supported(v)) ALLOC(m->eft, eloc_fast_table_bytes(v));
        if (lanczos_fast_supported(v)) ALLOC(m->lft, lanczos_fast_table_bytes(v));
    }
    if (d.precision == NNQS_BF16X2 || d.precision == NNQS_BF16X3) {
        const int ns = d.precision == NNQS_BF16X2 ? 2 : 3;
        if (tc_supported((int)N, d.M, m->G, d.K, m->nsign, ns)) {
            m->ns = ns;
            ALLOC(m->bimg, tc_bimg_bytes((int)N, d.M, m->G, d.K, m->nsign, ns));
            ALLOC(m->pinv, tc_pinv_bytes((int)N, m->G));
        }
    }
#undef ALLOC
    cudaMemcpy(m->perm, perm.data(), perm.size(), cudaMemcpyHostToDevice);
    if (m->pinv) {
        std::vector<uint16_t> inv(tc_pinv_bytes(m->N, m->G) / sizeof(uint16_t));
        tc_pinv_table(perm.data(), m->N, m->G, inv.data());
        cudaMemcpy(m->pinv, inv.data(), inv.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    }
    {
        // image of every bond under every group element, with the orientation flag
        std::vector<int> index((size_t)N * N, -1);
        for (size_t b = 0; b < bi.size(); ++b) {
            index[(size_t)bi[b] * N + bj[b]] = (int)b;
            index[(size_t)bj[b] * N + bi[b]] = (int)b;
        }
        std::vector<uint16_t> bp((size_t)m->G * bi.size());
        for (int g = 0; g < m->G; ++g)
            for (size_t b = 0; b < bi.size(); ++b) {
                const int gi = perm[(size_t)g * N + bi[b]], gj = perm[(size_t)g * N + bj[b]];
                const int img = index[(size_t)gi * N + gj];
                if (img < 0) return cleanup(fail(NNQS_EINVAL, "symmetry operation does not map bonds to bonds"));
                bp[(size_t)g * bi.size() + b] = (uint16_t)(img | (bi[img] != gi ? 0x8000 : 0));
            }
        cudaMemcpy(m->bperm, bp.data(), bp.size() * sizeof(uint16_t), cudaMemcpyHostToDevice);
    }
    cudaMemcpy(m->bi, bi.data(), bi.size() * 2, cudaMemcpyHostToDevice);
    cudaMemcpy(m->bj, bj.data(), bj.size() * 2, cudaMemcpyHostToDevice);
    cudaMemcpy(m->bt, bt.data(), bt.size(), cudaMemcpyHostToDevice);
    if (m->fp64) {
        cudaMemcpy(m->chi, chi.data(), chi.size() * 8, cudaMemcpyHostToDevice);
    } else {
        std::vector<float> cf(chi.begin(), chi.end());
        cudaMemcpy(m->chi, cf.data(), cf.size() * 4, cudaMemcpyHostToDevice);
    }
    cudaMemset(m->status, 0, sizeof(int));
    std::vector<double> zero((size_t)m->P * 2, 0.0);
    cudaError_t e = cudaMemcpy(m->params, zero.data(), zero.size() * 8, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "cudaMemcpy"));
    *out = m;
    return nnqs_set_params_device(m, m->params, m->P, nullptr) == NNQS_OK ? (cudaDeviceSynchronize(), NNQS_OK)
                                                                           : cleanup(NNQS_ECUDA);
}

int nnqs_create(const nnqs_desc *desc, nnqs_model **out) { return create_model(desc, 0, out); }

int nnqs_destroy(nnqs_model *m)
{
    if (!m) return NNQS_OK;
    cudaDeviceSynchronize();
    void *ptrs[] = {m->perm, m->bi, m->bj, m->bt, m->chi, m->params, m->Wt, m->b, m->a, m->logc, m->X, m->XA,
                    m->Tb, m->Cb, m->S4, m->CS, m->ES, m->bperm, m->status, m->chk, m->eft, m->lft, m->ws, m->bimg, m->pinv};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete m;
    return NNQS_OK;
}

int64_t nnqs_num_params(const nnqs_model *m) { return m ? m->P : -1; }
int32_t nnqs_group_size(const nnqs_model *m) { return m ? m->G : -1; }

int nnqs_set_params_device(nnqs_model *m, const double *params, int64_t P, void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    if (!params) return fail(NNQS_EINVAL, "params is NULL");
    if (P != m->P) return fail(NNQS_EINVAL, "expected %lld parameters, got %lld", (long long)m->P, (long long)P);
    return with_device(m, [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        if (params != m->params)
            NNQS_CUDA(cudaMemcpyAsync(m->params, params, (size_t)P * 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
        cudaError_t e;
        if (m->fp64)
            e = launch_build_tables<double>(m->params, m->N, m->d.M, m->d.K, (cx<double> *)m->Wt, (cx<double> *)m->b,
                                            (cx<double> *)m->a, (cx<double> *)m->logc, (cx2<double> *)m->X,
                                            (cx2<double> *)m->XA, st);
        else
            e = launch_build_tables<float>(m->params, m->N, m->d.M, m->d.K, (cx<float> *)m->Wt, (cx<float> *)m->b,
                                           (cx<float> *)m->a, (cx<float> *)m->logc, (cx2<float> *)m->X,
                                           (cx2<float> *)m->XA, st);
        if (e != cudaSuccess) return cuda_fail(e, "build tables");
        if (m->fp64)
            e = launch_tables_conn<double>(m->params, m->N, m->d.M, m->Mp, m->d.K, m->nbonds, m->d.use_bias, m->bi, m->bj,
                                           (cx<double> *)m->Tb, (cx<double> *)m->Cb, (cx<double> *)m->S4,
                                           (cx<double> *)m->CS, (sc<double> *)m->ES, st);
        else
            e = launch_tables_conn<float>(m->params, m->N, m->d.M, m->Mp, m->d.K, m->nbonds, m->d.use_bias, m->bi, m->bj,
                                          (cx<float> *)m->Tb, (cx<float> *)m->Cb, (cx<float> *)m->S4,
                                          (cx<float> *)m->CS, (sc<float> *)m->ES, st);
        if (e != cudaSuccess) return cuda_fail(e, "build connection tables");
        if (m->eft) {
            e = launch_tables_paired(view<float>(m), m->eft, st);
            if (e != cudaSuccess) return cuda_fail(e, "build paired tables");
        }
        if (m->lft) {
            e = launch_tables_site_paired(view<float>(m), m->lft, st);
            if (e != cudaSuccess) return cuda_fail(e, "build paired site tables");
        }
        if (m->ns) {
            e = launch_bimg(m->params, m->N, m->d.M, m->G, m->d.K, m->nsign, m->ns, m->d.use_bias, m->bimg, st);
            if (e != cudaSuccess) return cuda_fail(e, "build bf16 weight images");
        }
        return NNQS_OK;
    });
}

int nnqs_set_params(nnqs_model *m, const double *params, int64_t P, void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    if (!params) return fail(NNQS_EINVAL, "params is NULL");
    if (P != m->P) return fail(NNQS_EINVAL, "expected %lld parameters, got %lld", (long long)m->P, (long long)P);
    return with_device(m, [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        NNQS_CUDA(cudaMemcpyAsync(m->params, params, (size_t)P * 2 * sizeof(double), cudaMemcpyHostToDevice, st));
        NNQS_CUDA(cudaStreamSynchronize(st));  // the host buffer may be reused on return
        return nnqs_set_params_device(m, m->params, P, stream);
    });
}

int nnqs_log_psi(nnqs_model *m, const uint64_t *cfg, int64_t n, double *out, void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    if (n < 0) return fail(NNQS_EINVAL, "n < 0");
    if (n == 0) return NNQS_OK;
    if (!cfg || !out) return fail(NNQS_EINVAL, "cfg and logpsi_out must be non-NULL");
    return with_device(m, [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        if (int rc = check_cfg(m, cfg, n, st)) return rc;
        cudaError_t e;
        if (m->fp64) e = launch_log_psi(view<double>(m), cfg, n, out, m->nsm, st);
        else if (m->ns) e = launch_log_psi_tc(view<float>(m), m->bimg, m->pinv, m->ns, cfg, n, out, m->nsm, st);
        else e = launch_log_psi(view<float>(m), cfg, n, out, m->nsm, st);
        if (e == cudaSuccess) e = mark_vanishing(m, cfg, n, 0, out, nullptr, st);
        return e == cudaSuccess ? NNQS_OK : cuda_fail(e, "log_psi");
    });
}

int nnqs_local_energy(nnqs_model *m, const uint64_t *cfg, int64_t n, double *eloc, double *sums, void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    if (n < 0) return fail(NNQS_EINVAL, "n < 0");
    if (n == 0) return NNQS_OK;
    if (!cfg || !eloc) return fail(NNQS_EINVAL, "cfg and eloc_out must be non-NULL");
    return with_device(m, [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        if (int rc = check_cfg(m, cfg, n, st)) return rc;
        cudaError_t e;
        if (m->fp64) e = launch_ratio(view<double>(m), cfg, n, 0, eloc, nullptr, m->nsm, st);
        else if (m->eft && !test_old_engine()) e = launch_eloc_fast(view<float>(m), m->eft, cfg, n, eloc, m->nsm, st);
        else e = launch_ratio(view<float>(m), cfg, n, 0, eloc, nullptr, m->nsm, st);
        if (e == cudaSuccess) e = mark_vanishing(m, cfg, n, 1, eloc, nullptr, st);
        if (e != cudaSuccess) return cuda_fail(e, "local_energy");
        if (sums) {
            const int nb = 64;
            int rc = ensure_ws(m, nb * kMomentSums * sizeof(double));
            if (rc) return rc;
            e = launch_eloc_sums(eloc, n, (double *)m->ws, nb, sums, st);
            if (e != cudaSuccess) return cuda_fail(e, "eloc sums");
        }
        return NNQS_OK;
    });
}

int nnqs_lanczos_moments(nnqs_model *m, const uint64_t *cfg, int64_t n, double *h1, double *h2, double *moments,
                         double *lanczos, void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    if (n < 0) return fail(NNQS_EINVAL, "n < 0");
    if (n == 0) return NNQS_OK;
    if (!cfg) return fail(NNQS_EINVAL, "cfg must be non-NULL");
    return with_device(m, [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        const int nb = 64;
        if (int rc = check_cfg(m, cfg, n, st)) return rc;
        size_t need = align256(nb * kMomentSums * sizeof(double));
        const size_t off_h1 = need;
        if (!h1) need += align256((size_t)n * 2 * sizeof(double));
        const size_t off_h2 = need;
        if (!h2) need += align256((size_t)n * 2 * sizeof(double));
        int rc = ensure_ws(m, need);
        if (rc) return rc;
        char *ws = (char *)m->ws;
        double *H1 = h1 ? h1 : (double *)(ws + off_h1);
        double *H2 = h2 ? h2 : (double *)(ws + off_h2);
        cudaError_t e = lanczos_h(m, cfg, n, H1, H2, st);
        if (e == cudaSuccess) e = mark_vanishing(m, cfg, n, 1, H1, H2, st);
        if (e != cudaSuccess) return cuda_fail(e, "lanczos");
        if (moments || lanczos) {
            e = launch_moments(H1, H2, n, (double *)ws, nb, moments, lanczos, st);
            if (e != cudaSuccess) return cuda_fail(e, "moments");
        }
        return NNQS_OK;
    });
}

int nnqs_lanczos_partial(nnqs_model *m, const uint64_t *cfg, int64_t n, double *h1, double *h2, double *sums,
                         void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    if (n < 0) return fail(NNQS_EINVAL, "n < 0");
    if (!sums) return fail(NNQS_EINVAL, "sums_out must be non-NULL");
    if (n > 0 && !cfg) return fail(NNQS_EINVAL, "cfg must be non-NULL");
    return with_device(m, [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        if (n == 0) {
            NNQS_CUDA(cudaMemsetAsync(sums, 0, kMomentSums * sizeof(double), st));
            return NNQS_OK;
        }
        if (int rc = check_cfg(m, cfg, n, st)) return rc;
        const int nb = 64;
        size_t need = align256(nb * kMomentSums * sizeof(double));
        const size_t off_h1 = need;
        if (!h1) need += align256((size_t)n * 2 * sizeof(double));
        const size_t off_h2 = need;
        if (!h2) need += align256((size_t)n * 2 * sizeof(double));
        int rc = ensure_ws(m, need);
        if (rc) return rc;
        char *ws = (char *)m->ws;
        double *H1 = h1 ? h1 : (double *)(ws + off_h1);
        double *H2 = h2 ? h2 : (double *)(ws + off_h2);
        cudaError_t e = lanczos_h(m, cfg, n, H1, H2, st);
        if (e == cudaSuccess) e = mark_vanishing(m, cfg, n, 1, H1, H2, st);
        if (e == cudaSuccess) e = launch_moments(H1, H2, n, (double *)ws, nb, nullptr, nullptr, st, sums);
        return e == cudaSuccess ? NNQS_OK : cuda_fail(e, "lanczos_partial");
    });
}

int nnqs_lanczos_finish(const double *sums, double *moments, double *lanczos, void *stream)
{
    if (!sums) return fail(NNQS_EINVAL, "sums must be non-NULL");
    if (!moments && !lanczos) return NNQS_OK;
    const cudaError_t e = launch_moments_finish(sums, moments, lanczos, (cudaStream_t)stream);
    return e == cudaSuccess ? NNQS_OK : cuda_fail(e, "lanczos_finish");
}

int nnqs_sample(nnqs_model *m, uint64_t seed, int32_t n_chains, int32_t n_per_chain, int32_t n_skip, int32_t n_burn,
                uint64_t *cfg_out, float *acc_out, void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    if (n_chains <= 0 || n_per_chain <= 0 || n_skip <= 0 || n_burn < 0)
        return fail(NNQS_EINVAL, "n_chains, n_per_chain, n_skip must be > 0 and n_burn >= 0");
    if (!cfg_out) return fail(NNQS_EINVAL, "cfg_out must be non-NULL");
    if ((int64_t)n_burn + (int64_t)n_per_chain * n_skip > 0x7fffffffLL)
        return fail(NNQS_EINVAL, "total number of steps exceeds 2^31 - 1");
    return with_device(m, [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        if (!m->fp64) {
            // the chain caches in the shared memory of thread-block clusters, when they fit
            cudaError_t e = cudaSuccess;
            if (launch_sample_cl(view<float>(m), seed, n_chains, n_per_chain, n_skip, n_burn, cfg_out, acc_out, m->nsm,
                                 st, &e))
                return e == cudaSuccess ? NNQS_OK : cuda_fail(e, "sample (cluster)");
        }
        const size_t per = m->fp64 ? sampler_cache_bytes(view<double>(m)) : sampler_cache_bytes(view<float>(m));
        const int conc = m->fp64 ? sampler_grid(view<double>(m), n_chains, m->nsm) : sampler_grid(view<float>(m), n_chains, m->nsm);
        (void)conc;
        int rc = ensure_ws(m, per * (size_t)n_chains);
        if (rc) return rc;
        cudaError_t e = m->fp64
                            ? launch_sample(view<double>(m), seed, n_chains, n_per_chain, n_skip, n_burn, cfg_out, acc_out, m->ws, m->nsm, st)
                            : launch_sample(view<float>(m), seed, n_chains, n_per_chain, n_skip, n_burn, cfg_out, acc_out, m->ws, m->nsm, st);
        return e == cudaSuccess ? NNQS_OK : cuda_fail(e, "sample");
    });
}

int nnqs_grad_logpsi(nnqs_model *m, const uint64_t *cfg, int64_t n, double *O, void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    if (n < 0) return fail(NNQS_EINVAL, "n < 0");
    if (n == 0) return NNQS_OK;
    if (!cfg || !O) return fail(NNQS_EINVAL, "cfg and O_out must be non-NULL");
    if ((size_t)m->G * m->N > 200 * 1024) return fail(NNQS_EUNSUPPORTED, "|G| * N too large for the gradient kernel");
    return with_device(m, [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        if (int rc = check_cfg(m, cfg, n, st)) return rc;
        cudaError_t e;
        if (m->fp64) {
            const DevModel<double> v = view<double>(m);
            const int grid = grad_grid(v, n, m->nsm);
            int rc = ensure_ws(m, grad_scratch_bytes(v) * grid);
            if (rc) return rc;
            e = launch_grad(v, cfg, n, O, m->ws, grid, st);
        } else {
            const DevModel<float> v = view<float>(m);
            const int grid = grad_grid(v, n, m->nsm);
            const size_t gs = align256(grad_scratch_bytes(v) * grid);
            // tensor-core models: theta' of a chunk of samples from the tcgen05
            // GEMM (at most 4 GiB of [K][G][M] float2 rows at a time), then the
            // gradient kernel reads it
            const size_t per = (size_t)v.K * v.G * v.M * sizeof(float2);
            int64_t cs = 0;
            if (m->ns) cs = std::max<int64_t>(1, std::min<int64_t>(n, (int64_t)(((size_t)4 << 30) / per)));
            int rc = ensure_ws(m, gs + (size_t)cs * per);
            if (rc) return rc;
            if (!cs) {
                e = launch_grad(v, cfg, n, O, m->ws, grid, st);
            } else {
                float2 *th = reinterpret_cast<float2 *>((char *)m->ws + gs);
                e = cudaSuccess;
                for (int64_t c0 = 0; c0 < n && e == cudaSuccess; c0 += cs) {
                    const int64_t k = std::min<int64_t>(cs, n - c0);
                    const uint64_t *c = cfg + c0 * m->nwords;
                    e = launch_log_psi_tc(v, m->bimg, m->pinv, m->ns, c, k, nullptr, m->nsm, st, th);
                    if (e == cudaSuccess) e = launch_grad(v, c, k, O + c0 * m->P * 2, m->ws, grad_grid(v, k, m->nsm), st, th);
                }
            }
        }
        return e == cudaSuccess ? NNQS_OK : cuda_fail(e, "grad_logpsi");
    });
}

int nnqs_energy_grad(const nnqs_model *mc, const double *O, const double *eloc, const double *weights, int64_t n,
                     double *F, void *stream)
{
    nnqs_model *m = const_cast<nnqs_model *>(mc);
    if (check_model(m)) return NNQS_EINVAL;
    if (n <= 0) return fail(NNQS_EINVAL, "n must be > 0");
    if (!O || !eloc || !F) return fail(NNQS_EINVAL, "O, eloc and F_out must be non-NULL");
    if ((uintptr_t)O & 15) return fail(NNQS_EINVAL, "O must be 16-byte aligned");
    return with_device(m, [&]() -> int {
        int rc = ensure_ws(m, egrad_scratch_doubles(n, m->P) * sizeof(double));
        if (rc) return rc;
        cudaError_t e = launch_energy_grad(O, eloc, weights, n, m->P, F, (double *)m->ws, (cudaStream_t)stream);
        return e == cudaSuccess ? NNQS_OK : cuda_fail(e, "energy_grad");
    });
}

int nnqs_sr_matvec(const nnqs_model *mc, const double *O, const double *weights, int64_t n, const double *x,
                   double lambda, double *y, void *stream)
{
    nnqs_model *m = const_cast<nnqs_model *>(mc);
    if (check_model(m)) return NNQS_EINVAL;
    if (n <= 0) return fail(NNQS_EINVAL, "n must be > 0");
    if (!O || !x || !y) return fail(NNQS_EINVAL, "O, x and y must be non-NULL");
    if (((uintptr_t)O | (uintptr_t)x) & 15) return fail(NNQS_EINVAL, "O and x must be 16-byte aligned");
    return with_device(m, [&]() -> int {
        int rc = ensure_ws(m, sr_scratch_doubles(n, m->P) * sizeof(double));
        if (rc) return rc;
        cudaError_t e = launch_sr_matvec(O, weights, n, m->P, x, lambda, y, (double *)m->ws, (cudaStream_t)stream);
        return e == cudaSuccess ? NNQS_OK : cuda_fail(e, "sr_matvec");
    });
}

int nnqs_sr_solve(const nnqs_model *mc, const double *O, const double *weights, int64_t n, const double *F,
                  double lambda, double dtau, int32_t max_iter, double tol, double *delta, double *info,
                  double *params_inout, void *stream)
{
    nnqs_model *m = const_cast<nnqs_model *>(mc);
    if (check_model(m)) return NNQS_EINVAL;
    if (n <= 0) return fail(NNQS_EINVAL, "n must be > 0");
    if (max_iter < 0 || max_iter > 100000) return fail(NNQS_EINVAL, "max_iter must be in 0..100000");
    if (!(lambda >= 0) || !(tol >= 0)) return fail(NNQS_EINVAL, "lambda and tol must be >= 0");
    if (!O || !F || !delta) return fail(NNQS_EINVAL, "O, F and delta_out must be non-NULL");
    if ((uintptr_t)O & 15) return fail(NNQS_EINVAL, "O must be 16-byte aligned");
    return with_device(m, [&]() -> int {
        int rc = ensure_ws(m, sr_scratch_doubles(n, m->P) * sizeof(double));
        if (rc) return rc;
        cudaError_t e = launch_sr_solve(O, weights, n, m->P, F, lambda, dtau, max_iter, tol, delta, info,
                                        params_inout, (double *)m->ws, (cudaStream_t)stream);
        return e == cudaSuccess ? NNQS_OK : cuda_fail(e, "sr_solve");
    });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Fixed-size scratch of nnqs_lanczos_moments_noalloc: h1 [max][2], h2 [max][2]
// and the FP64 partial sums [kNoallocBlocks][kMomentSums].  In host code the array's
// name is only a stand-in; its device address is looked up once per device.
// ---------------------------------------------------------------------------
namespace {
constexpr int kNoallocBlocks = 64;
constexpr size_t kNoallocDoubles = (size_t)4 * NNQS_NOALLOC_MAX_SAMPLES + (size_t)kNoallocBlocks * kMomentSums;
}  // namespace

static __device__ __align__(256) double g_noalloc_scratch[kNoallocDoubles];

namespace {
std::mutex g_noalloc_mu;
double *g_noalloc_ptr[128] = {};  // device address of g_noalloc_scratch, per device

int noalloc_scratch(int device, double **out)
{
    if (device < 0 || device >= 128) return fail(NNQS_EUNSUPPORTED, "device ordinal %d out of range", device);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[device]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // current device == device
        if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
        g_noalloc_ptr[device] = (double *)p;
    }
    *out = g_noalloc_ptr[device];
    return NNQS_OK;
}
}  // namespace

extern "C" {

int nnqs_lanczos_moments_noalloc(nnqs_model *m, const uint64_t *cfg, int64_t n, double *moments, double *lanczos,
                                 void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    if (n < 0) return fail(NNQS_EINVAL, "n < 0");
    if (n > NNQS_NOALLOC_MAX_SAMPLES)
        return fail(NNQS_EINVAL, "n = %lld exceeds the fixed scratch of %d samples", (long long)n,
                    NNQS_NOALLOC_MAX_SAMPLES);
    if (n == 0) return NNQS_OK;
    if (!cfg) return fail(NNQS_EINVAL, "cfg must be non-NULL");
    return with_device(m, [&]() -> int {
        double *base = nullptr;
        const int rc = noalloc_scratch(m->device, &base);
        if (rc) return rc;
        double *h1 = base, *h2 = base + 2 * (size_t)NNQS_NOALLOC_MAX_SAMPLES;
        double *partial = base + 4 * (size_t)NNQS_NOALLOC_MAX_SAMPLES;
        cudaStream_t st = (cudaStream_t)stream;
        if (int rc = check_cfg(m, cfg, n, st)) return rc;
        cudaError_t e = lanczos_h(m, cfg, n, h1, h2, st);
        if (e == cudaSuccess) e = mark_vanishing(m, cfg, n, 1, h1, h2, st);
        if (e != cudaSuccess) return cuda_fail(e, "lanczos (fixed scratch)");
        if (moments || lanczos) {
            e = launch_moments(h1, h2, n, partial, kNoallocBlocks, moments, lanczos, st);
            if (e != cudaSuccess) return cuda_fail(e, "moments (fixed scratch)");
        }
        return NNQS_OK;
    });
}

int nnqs_lanczos2(nnqs_model *m, const uint64_t *cfg, int64_t n, double *h3_out, double *mu_out, double *out,
                  void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    if (n < 1) return fail(NNQS_EINVAL, "n must be >= 1");
    if (!cfg) return fail(NNQS_EINVAL, "cfg must be non-NULL");
    const int64_t tmax = n * (int64_t)m->nbonds;  // at most one neighbour per bond
    if (tmax > 0x7fffffffLL) return fail(NNQS_EINVAL, "too many neighbour configurations (n x 4N >= 2^31)");
    return with_device(m, [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        if (int rc = check_cfg(m, cfg, n, st)) return rc;
        // workspace: every piece 256-byte aligned, sized for the upper bound of neighbours
        size_t at = 0;
        auto take = [&](size_t bytes) { const size_t o = at; at += align256(bytes); return o; };
        const size_t o_cnt = take(n * 8), o_off = take((n + 1) * 8);
        const size_t o_h1 = take(n * 16), o_h2 = take(n * 16), o_h3 = take(n * 16), o_lp = take(n * 16);
        const size_t o_part = take(64 * kMomentSums * 8), o_mom = take(8 * 8), o_part2 = take(kShiftBlocks * 8 * 8);
        const size_t o_ncfg = take((size_t)tmax * m->nwords * 8), o_ncoef = take((size_t)tmax * 8);
        const size_t o_lpn = take((size_t)tmax * 16), o_h1n = take((size_t)tmax * 16), o_h2n = take((size_t)tmax * 16);
        int rc = ensure_ws(m, at);
        if (rc) return rc;
        char *ws = (char *)m->ws;
        int64_t *cnt = (int64_t *)(ws + o_cnt), *off = (int64_t *)(ws + o_off);
        double *h1 = (double *)(ws + o_h1), *h2 = (double *)(ws + o_h2), *lp = (double *)(ws + o_lp);
        double *h3 = h3_out ? h3_out : (double *)(ws + o_h3);
        double *part = (double *)(ws + o_part), *mom = (double *)(ws + o_mom), *part2 = (double *)(ws + o_part2);
        uint64_t *ncfg = (uint64_t *)(ws + o_ncfg);
        double *ncoef = (double *)(ws + o_ncoef), *lpn = (double *)(ws + o_lpn);
        double *h1n = (double *)(ws + o_h1n), *h2n = (double *)(ws + o_h2n);
        cudaError_t e = m->fp64 ? launch_expand_nb(view<double>(m), cfg, n, cnt, off, st)
                                : launch_expand_nb(view<float>(m), cfg, n, cnt, off, st);
        if (e != cudaSuccess) return cuda_fail(e, "neighbour count");
        int64_t T = 0;
        NNQS_CUDA(cudaMemcpyAsync(&T, off + n, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        NNQS_CUDA(cudaStreamSynchronize(st));
        if (T < 0 || T > tmax) return fail(NNQS_ECUDA, "neighbour count %lld out of range", (long long)T);
        auto log_psi = [&](const uint64_t *c, int64_t k, double *o) -> cudaError_t {
            if (k == 0) return cudaSuccess;
            cudaError_t e2;
            if (m->fp64) e2 = launch_log_psi(view<double>(m), c, k, o, m->nsm, st);
            else if (m->ns) e2 = launch_log_psi_tc(view<float>(m), m->bimg, m->pinv, m->ns, c, k, o, m->nsm, st);
            else e2 = launch_log_psi(view<float>(m), c, k, o, m->nsm, st);
            return e2 == cudaSuccess ? mark_vanishing(m, c, k, 0, o, nullptr, st) : e2;
        };
        auto ratio = [&](const uint64_t *c, int64_t k, double *a, double *b) -> cudaError_t {
            if (k == 0) return cudaSuccess;
            const cudaError_t e2 = lanczos_h(m, c, k, a, b, st);
            return e2 == cudaSuccess ? mark_vanishing(m, c, k, 1, a, b, st) : e2;
        };
        e = m->fp64 ? launch_fill_nb(view<double>(m), cfg, n, off, ncfg, ncoef, st)
                    : launch_fill_nb(view<float>(m), cfg, n, off, ncfg, ncoef, st);
        if (e == cudaSuccess) e = log_psi(cfg, n, lp);
        if (e == cudaSuccess) e = log_psi(ncfg, T, lpn);
        if (e == cudaSuccess) e = ratio(cfg, n, h1, h2);
        if (e == cudaSuccess) e = ratio(ncfg, T, h1n, h2n);
        if (e == cudaSuccess)
            e = m->fp64 ? launch_h3(view<double>(m), cfg, n, off, ncoef, lp, lpn, h2, h2n, h3, st)
                        : launch_h3(view<float>(m), cfg, n, off, ncoef, lp, lpn, h2, h2n, h3, st);
        if (e != cudaSuccess) return cuda_fail(e, "lanczos2 (h3)");
        if (mu_out || out) {
            e = launch_moments(h1, h2, n, part, 64, mom, nullptr, st);  // c = mom[1] = <Re h1>
            if (e == cudaSuccess) e = launch_krylov2(h1, h2, h3, n, mom + 1, part2, kShiftBlocks, mu_out, out, st);
            if (e != cudaSuccess) return cuda_fail(e, "lanczos2 (moments)");
        }
        return NNQS_OK;
    });
}

int nnqs_lanczos_variance(const double *moments, const double *lanczos, double *out, void *stream)
{
    if (!moments || !lanczos || !out) return fail(NNQS_EINVAL, "moments, lanczos and out must be non-NULL");
    const cudaError_t e = launch_lanczos_variance(moments, lanczos, out, (cudaStream_t)stream);
    return e == cudaSuccess ? NNQS_OK : cuda_fail(e, "lanczos_variance");
}

int nnqs_structure_factor(nnqs_model *m, const uint64_t *cfg, int64_t n, const double *weights, double *sq_out,
                          void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    if (n < 1) return fail(NNQS_EINVAL, "n must be >= 1");
    if (!cfg || !sq_out) return fail(NNQS_EINVAL, "cfg and sq_out must be non-NULL");
    return with_device(m, [&]() -> int {
        if (int rc = check_cfg(m, cfg, n, (cudaStream_t)stream)) return rc;
        const int grid = sq_grid(n, m->nsm);
        int rc = ensure_ws(m, (size_t)grid * (m->N + 1) * sizeof(double));
        if (rc) return rc;
        const cudaError_t e = launch_structure_factor(cfg, n, m->d.L, m->nwords, weights, (double *)m->ws, grid,
                                                      sq_out, (cudaStream_t)stream);
        return e == cudaSuccess ? NNQS_OK : cuda_fail(e, "structure_factor");
    });
}

int nnqs_status(nnqs_model *m, void *stream)
{
    if (check_model(m)) return NNQS_EINVAL;
    return with_device(m, [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        int h = 0;
        NNQS_CUDA(cudaStreamSynchronize(st));
        NNQS_CUDA(cudaMemcpy(&h, m->status, sizeof(int), cudaMemcpyDeviceToHost));
        NNQS_CUDA(cudaMemset(m->status, 0, sizeof(int)));
        if (h == NNQS_ETIMEOUT) return fail(h, "a bounded device-side wait ran out (the kernel returned early)");
        if (h) return fail(h, "a kernel produced a non-finite amplitude");
        return NNQS_OK;
    });
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Mixed batch: instances of uneven size in one persistent launch
// ---------------------------------------------------------------------------
struct nnqs_batch {
    std::vector<nnqs_model *> models;
    std::vector<int> shape;     // tile shape of each instance (index into kTileGL / kTileMPL)
    std::vector<double> cost;   // per-sample work estimate, orders the work list
    int device = 0, nsm = 0, grid = 0;
    DevModel<float> *d_models = nullptr;
    int *d_shape = nullptr, *d_counter = nullptr;
    int64_t *d_cfg_off = nullptr, *d_out_off = nullptr;
    BatchItem *d_items = nullptr, *d_titems = nullptr;
    size_t items_cap = 0, titems_cap = 0;
    double *d_h = nullptr, *d_th = nullptr;  // h1 | h2 when the caller passes none; tuning outputs
    size_t h_cap = 0, th_cap = 0;
    cudaStream_t cap = nullptr;
    cudaGraphExec_t exec = nullptr;
    // arguments the captured graph was built for
    const uint64_t *k_cfg = nullptr;
    double *k_h1 = nullptr, *k_h2 = nullptr, *k_mo = nullptr, *k_lz = nullptr;
    std::vector<int64_t> k_n;
};

namespace {

int shape_width(int v) { return kTileGL[v] * kTileMPL[v]; }

// Tile shapes an instance of width M may run with: every shape from the
// narrowest width that holds M up to 15% wider.
std::vector<int> shape_candidates(int M)
{
    int w0 = 1 << 30;
    for (int v = 0; v < kNumTileShapes; ++v)
        if (shape_width(v) >= M && shape_width(v) < w0) w0 = shape_width(v);
    const int wmax = w0 + (w0 * 15 + 99) / 100;
    std::vector<int> c;
    for (int v = 0; v < kNumTileShapes; ++v)
        if (shape_width(v) >= M && shape_width(v) <= wmax) c.push_back(v);
    return c;
}

int widest(const std::vector<int> &c)
{
    int w = 0;
    for (int v : c) w = shape_width(v) > w ? shape_width(v) : w;
    return w;
}

template <typename P> int grow(P *&p, size_t &cap, size_t n)
{
    if (n <= cap) return NNQS_OK;
    if (p) {
        cudaDeviceSynchronize();
        cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    cudaError_t e = cudaMalloc((void **)&p, n * sizeof(P));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(NNQS_ENOMEM, "batch buffer of %zu bytes refused", n * sizeof(P));
    }
    cap = n;
    return NNQS_OK;
}

void drop_graph(nnqs_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
    b->k_n.clear();
}

int batch_check(const nnqs_batch *b, const uint64_t *cfg, const int64_t *n, int64_t &total)
{
    if (!b) return fail(NNQS_EINVAL, "batch is NULL");
    if (!n) return fail(NNQS_EINVAL, "n_per_model must be non-NULL");
    total = 0;
    for (size_t i = 0; i < b->models.size(); ++i) {
        if (n[i] < 0) return fail(NNQS_EINVAL, "n_per_model[%zu] < 0", i);
        total += n[i];
    }
    if (total > 0x7fffffffLL) return fail(NNQS_EINVAL, "more than 2^31 - 1 samples in one batch");
    if (total > 0 && !cfg) return fail(NNQS_EINVAL, "cfg must be non-NULL");
    return NNQS_OK;
}

void batch_offsets(const nnqs_batch *b, const int64_t *n, std::vector<int64_t> &cfg_off, std::vector<int64_t> &out_off)
{
    const size_t nm = b->models.size();
    cfg_off.assign(nm, 0);
    out_off.assign(nm + 1, 0);
    for (size_t i = 0; i < nm; ++i) {
        if (i) cfg_off[i] = cfg_off[i - 1] + n[i - 1] * b->models[i - 1]->nwords;
        out_off[i + 1] = out_off[i] + n[i];
    }
}

// Checked mode of the instances that asked for it (desc.check_inputs).
int batch_check_cfg(const nnqs_batch *b, const uint64_t *cfg, const int64_t *n, cudaStream_t st)
{
    std::vector<int64_t> cfg_off, out_off;
    batch_offsets(b, n, cfg_off, out_off);
    for (size_t i = 0; i < b->models.size(); ++i) {
        if (int rc = check_cfg(b->models[i], cfg + cfg_off[i], n[i], st))
            return fail(rc, "instance %zu: %s", i, std::string(g_err).c_str());
    }
    return NNQS_OK;
}

}  // namespace

extern "C" {

int32_t nnqs_num_tile_shapes(void) { return kNumTileShapes; }

int nnqs_tile_shape(int32_t v, int32_t *gl, int32_t *mpl)
{
    if (v < 0 || v >= kNumTileShapes) return fail(NNQS_EINVAL, "tile shape %d out of range", v);
    if (gl) *gl = kTileGL[v];
    if (mpl) *mpl = kTileMPL[v];
    return NNQS_OK;
}

int nnqs_batch_destroy(nnqs_batch *b)
{
    if (!b) return NNQS_OK;
    cudaDeviceSynchronize();
    drop_graph(b);
    for (nnqs_model *m : b->models) nnqs_destroy(m);
    void *ptrs[] = {b->d_models, b->d_shape, b->d_counter, b->d_cfg_off, b->d_out_off,
                    b->d_items, b->d_titems, b->d_h, b->d_th};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (b->cap) cudaStreamDestroy(b->cap);
    delete b;
    return NNQS_OK;
}

int nnqs_batch_create(const nnqs_desc *descs, int32_t n_models, nnqs_batch **out)
{
    if (!descs || !out) return fail(NNQS_EINVAL, "descs and out must be non-NULL");
    *out = nullptr;
    if (n_models < 1) return fail(NNQS_EINVAL, "n_models must be >= 1");
    for (int i = 0; i < n_models; ++i)
        if (descs[i].precision == NNQS_FP64)
            return fail(NNQS_EUNSUPPORTED, "instance %d: the mixed batch runs the FP32 engine (precision FP64)", i);
    nnqs_batch *b = new nnqs_batch();
    auto cleanup = [&](int rc) { nnqs_batch_destroy(b); return rc; };
    cudaGetDevice(&b->device);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device);
    std::vector<DevModel<float>> views;
    for (int i = 0; i < n_models; ++i) {
        const std::vector<int> c = shape_candidates(descs[i].M);
        nnqs_model *m = nullptr;
        int rc = create_model(&descs[i], widest(c), &m);
        if (rc) return cleanup(rc);
        b->models.push_back(m);
        b->shape.push_back(c.front());
        // Lanczos work per sample ~ (pairs of exchanged bonds) x rows x width
        const double nb = 2.0 * m->N;
        b->cost.push_back(nb * nb * (double)m->d.K * m->G * m->nsign * shape_width(c.front()));
        views.push_back(view<float>(m));
    }
    b->grid = mixed_grid(b->nsm);
    if (b->grid <= 0) return cleanup(fail(NNQS_ECUDA, "mixed-batch kernel cannot be resident"));
#define BALLOC(ptr, count)                                                                       \
    do {                                                                                         \
        cudaError_t e_ = cudaMalloc((void **)&(ptr), sizeof(*(ptr)) * (size_t)(count));          \
        if (e_ != cudaSuccess) { cudaGetLastError(); return cleanup(cuda_fail(e_, "cudaMalloc")); } \
    } while (0)
    BALLOC(b->d_models, n_models);
    BALLOC(b->d_shape, n_models);
    BALLOC(b->d_counter, 1);
    BALLOC(b->d_cfg_off, n_models);
    BALLOC(b->d_out_off, n_models + 1);
#undef BALLOC
    cudaError_t e = cudaMemcpy(b->d_models, views.data(), views.size() * sizeof(DevModel<float>), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->d_shape, b->shape.data(), b->shape.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "batch setup"));
    *out = b;
    return NNQS_OK;
}

int32_t nnqs_batch_size(const nnqs_batch *b) { return b ? (int32_t)b->models.size() : -1; }

nnqs_model *nnqs_batch_model(nnqs_batch *b, int32_t i)
{
    if (!b || i < 0 || i >= (int32_t)b->models.size()) {
        fail(NNQS_EINVAL, "instance index out of range");
        return nullptr;
    }
    return b->models[i];
}

int32_t nnqs_batch_get_shape(const nnqs_batch *b, int32_t i)
{
    if (!b || i < 0 || i >= (int32_t)b->models.size()) return -1;
    return b->shape[i];
}

int nnqs_batch_set_shape(nnqs_batch *b, int32_t i, int32_t v)
{
    if (!b || i < 0 || i >= (int32_t)b->models.size()) return fail(NNQS_EINVAL, "instance index out of range");
    if (v < 0 || v >= kNumTileShapes) return fail(NNQS_EINVAL, "tile shape %d out of range", v);
    const nnqs_model *m = b->models[i];
    if (shape_width(v) < m->d.M || shape_width(v) > m->Mp)
        return fail(NNQS_EINVAL, "tile shape %d (width %d) does not fit instance %d (M = %d, table stride %d)", v,
                    shape_width(v), i, m->d.M, m->Mp);
    return with_device(m, [&]() -> int {
        NNQS_CUDA(cudaDeviceSynchronize());
        NNQS_CUDA(cudaMemcpy(b->d_shape + i, &v, sizeof(int), cudaMemcpyHostToDevice));
        b->shape[i] = v;
        return NNQS_OK;
    });
}

int nnqs_batch_lanczos(nnqs_batch *b, const uint64_t *cfg, const int64_t *n_per_model, double *h1_out,
                       double *h2_out, double *moments_out, double *lanczos_out, void *stream)
{
    int64_t total = 0;
    if (int rc = batch_check(b, cfg, n_per_model, total)) return rc;
    const size_t nm = b->models.size();
    return with_device(b->models[0], [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        if (int rc = batch_check_cfg(b, cfg, n_per_model, st)) return rc;
        if (!h1_out || !h2_out) {
            if (int rc = grow(b->d_h, b->h_cap, (size_t)4 * (total > 0 ? total : 1))) return rc;
        }
        double *H1 = h1_out ? h1_out : b->d_h;
        double *H2 = h2_out ? h2_out : b->d_h + 2 * total;
        const std::vector<int64_t> nv(n_per_model, n_per_model + nm);
        const bool same = b->exec && b->k_cfg == cfg && b->k_h1 == H1 && b->k_h2 == H2 && b->k_mo == moments_out &&
                          b->k_lz == lanczos_out && b->k_n == nv;
        if (!same) {
            drop_graph(b);
            std::vector<int64_t> cfg_off, out_off;
            batch_offsets(b, n_per_model, cfg_off, out_off);
            // work list: instances in decreasing per-sample work, so that the
            // longest items are taken first and short ones fill the tail
            std::vector<int> order(nm);
            for (size_t i = 0; i < nm; ++i) order[i] = (int)i;
            std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->cost[x] > b->cost[y]; });
            std::vector<BatchItem> items;
            items.reserve((size_t)total);
            for (int i : order)
                for (int64_t k = 0; k < n_per_model[i]; ++k)
                    items.push_back(BatchItem{i, (int)k, (int)(out_off[i] + k)});
            if (int rc = grow(b->d_items, b->items_cap, items.size() > 0 ? items.size() : 1)) return rc;
            NNQS_CUDA(cudaStreamSynchronize(st));
            NNQS_CUDA(cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
            NNQS_CUDA(cudaMemcpy(b->d_cfg_off, cfg_off.data(), nm * sizeof(int64_t), cudaMemcpyHostToDevice));
            NNQS_CUDA(cudaMemcpy(b->d_out_off, out_off.data(), (nm + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
            // capture: reset the work counter, the persistent launch, the reduction
            cudaGraph_t g = nullptr;
            NNQS_CUDA(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
            cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), b->cap);
            if (e == cudaSuccess)
                e = launch_mixed(b->grid, b->d_models, b->d_shape, b->d_items, (int)total, b->d_counter, cfg,
                                 b->d_cfg_off, H1, H2, b->cap);
            if (e == cudaSuccess && (moments_out || lanczos_out))
                e = launch_moments_batched(H1, H2, b->d_out_off, (int)nm, moments_out, lanczos_out, b->cap);
            const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
            if (e == cudaSuccess) e = e2;
            if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
            if (g) cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                b->exec = nullptr;
                return cuda_fail(e, "capture of the mixed-batch graph");
            }
            b->k_cfg = cfg; b->k_h1 = H1; b->k_h2 = H2; b->k_mo = moments_out; b->k_lz = lanczos_out; b->k_n = nv;
        }
        NNQS_CUDA(cudaGraphLaunch(b->exec, st));
        return NNQS_OK;
    });
}

int nnqs_batch_autotune(nnqs_batch *b, const uint64_t *cfg, const int64_t *n_per_model, int32_t probe,
                        int32_t *shape_out, double *ms_out, void *stream)
{
    int64_t total = 0;
    if (int rc = batch_check(b, cfg, n_per_model, total)) return rc;
    if (probe < 1) return fail(NNQS_EINVAL, "probe must be >= 1");
    const size_t nm = b->models.size();
    return with_device(b->models[0], [&]() -> int {
        cudaStream_t st = (cudaStream_t)stream;
        if (int rc = batch_check_cfg(b, cfg, n_per_model, st)) return rc;
        std::vector<int64_t> cfg_off, out_off;
        batch_offsets(b, n_per_model, cfg_off, out_off);
        const int R = b->grid;  // one item per resident CTA: a full-load wave
        if (int rc = grow(b->d_titems, b->titems_cap, (size_t)R)) return rc;
        if (int rc = grow(b->d_th, b->th_cap, (size_t)4 * R)) return rc;
        NNQS_CUDA(cudaStreamSynchronize(st));
        NNQS_CUDA(cudaMemcpy(b->d_cfg_off, cfg_off.data(), nm * sizeof(int64_t), cudaMemcpyHostToDevice));
        cudaEvent_t e0, e1;
        NNQS_CUDA(cudaEventCreate(&e0));
        NNQS_CUDA(cudaEventCreate(&e1));
        struct Done { int N, M, G, nsign, bias, shape; double ms; };
        std::vector<Done> done;  // instances of the same size share a result
        // tune the smallest-K instance of each size first
        std::vector<int> order(nm);
        for (size_t i = 0; i < nm; ++i) order[i] = (int)i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return b->models[x]->d.K < b->models[y]->d.K; });
        std::vector<double> ms(nm, 0.0);
        int rc = NNQS_OK;
        for (int i : order) {
            const nnqs_model *m = b->models[i];
            const std::vector<int> cand = shape_candidates(m->d.M);
            if (cand.size() == 1) b->shape[i] = cand.front();
            if (cand.size() == 1 || n_per_model[i] == 0) continue;
            bool reused = false;
            for (const Done &d : done)
                if (d.N == m->N && d.M == m->d.M && d.G == m->G && d.nsign == m->nsign && d.bias == m->d.use_bias) {
                    b->shape[i] = d.shape; ms[i] = d.ms; reused = true;
                    break;
                }
            if (reused) continue;
            const int ns = (int)(n_per_model[i] < probe ? n_per_model[i] : probe);
            std::vector<BatchItem> items(R);
            for (int k = 0; k < R; ++k) items[k] = BatchItem{i, k % ns, k};
            cudaError_t e = cudaMemcpy(b->d_titems, items.data(), R * sizeof(BatchItem), cudaMemcpyHostToDevice);
            double best = 1e300;
            int best_v = cand.front();
            for (int v : cand) {
                if (e != cudaSuccess) break;
                e = cudaMemcpy(b->d_shape + i, &v, sizeof(int), cudaMemcpyHostToDevice);
                double t_min = 1e300;
                for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
                    e = cudaMemsetAsync(b->d_counter, 0, sizeof(int), st);
                    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                    if (e == cudaSuccess)
                        e = launch_mixed(b->grid, b->d_models, b->d_shape, b->d_titems, R, b->d_counter, cfg,
                                         b->d_cfg_off, b->d_th, b->d_th + 2 * R, st);
                    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                    float t = 0.f;
                    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                    if (e != cudaSuccess) break;
                    if (rep > 0 || t > 50.f) t_min = t < t_min ? t : t_min;  // first run warms up short ones
                    if (t > 50.f) break;                                     // long runs: one is enough
                }
                if (t_min < best) { best = t_min; best_v = v; }
            }
            if (e != cudaSuccess) { rc = cuda_fail(e, "autotune"); break; }
            b->shape[i] = best_v;
            ms[i] = best;
            done.push_back(Done{m->N, m->d.M, m->G, m->nsign, m->d.use_bias, best_v, best});
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc) return rc;
        NNQS_CUDA(cudaMemcpy(b->d_shape, b->shape.data(), nm * sizeof(int), cudaMemcpyHostToDevice));
        for (size_t i = 0; i < nm; ++i) {
            if (shape_out) shape_out[i] = b->shape[i];
            if (ms_out) ms_out[i] = ms[i];
        }
        return NNQS_OK;
    });
}

int nnqs_batch_status(nnqs_batch *b, void *stream)
{
    if (!b) return fail(NNQS_EINVAL, "batch is NULL");
    int worst = NNQS_OK;
    for (nnqs_model *m : b->models) {
        const int rc = nnqs_status(m, stream);
        if (rc != NNQS_OK && worst == NNQS_OK) worst = rc;
    }
    return worst;
}

}  // extern "C"
