// Plan construction: the precomputation that the paper's NTT class performs
// at initialisation (Section 3: roots of unity and their precomputed
// factors), done once per (N, moduli) on the host and uploaded to HBM.
//
// Tables per limb (Section 2.2):
//   fwd[k] = {psi^brv(k), floor(psi^brv(k) * beta / q)}    Cooley-Tukey twiddles
//   inv[k] = {psi^-brv(k), floor(psi^-brv(k) * beta / q)}  Gentleman-Sande twiddles
// with beta = 2^64 for wide limbs and 2^32 for narrow limbs (q < 2^30), the
// Shoup factor W' of the Harvey butterflies.  Entry 0 is never read; it holds 1.
//
// Cyclic plans (the cyclic NTT of Section 2.2, over a primitive N-th root
// omega) use the same transforms with the twist removed: for k = 2^s + i,
// i < 2^s, the negacyclic entry psi^brv(k) = psi^(N/2^(s+1)) (psi^2)^(brv_s(i)
// N/2^(s+1)) becomes omega^(brv_s(i) N/2^(s+1)).  The same butterfly loops
// then give the cyclic NTT in bit-reversed order and its inverse.
#include <string.h>

#include <algorithm>
#include <map>
#include <thread>
#include <tuple>

#include "hx_internal.h"

typedef unsigned __int128 u128;

namespace hx {

static inline uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) {
    return (uint64_t)(((u128)a * b) % q);
}

uint64_t powmod_u64(uint64_t a, uint64_t e, uint64_t q) {
    uint64_t r = 1 % q;
    a %= q;
    while (e) {
        if (e & 1) r = mulmod(r, a, q);
        a = mulmod(a, a, q);
        e >>= 1;
    }
    return r;
}

// Deterministic Miller-Rabin; these twelve bases decide every n < 3.3e24.
bool is_prime_u64(uint64_t n) {
    static const uint64_t B[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
    if (n < 2) return false;
    for (uint64_t p : B)
        if (n % p == 0) return n == p;
    uint64_t d = n - 1;
    int s = 0;
    while (!(d & 1)) { d >>= 1; ++s; }
    for (uint64_t a : B) {
        uint64_t x = powmod_u64(a, d, n);
        if (x == 1 || x == n - 1) continue;
        bool composite = true;
        for (int r = 1; r < s && composite; ++r) {
            x = mulmod(x, x, n);
            if (x == n - 1) composite = false;
        }
        if (composite) return false;
    }
    return true;
}

// Smallest primitive 2N-th root of unity mod prime q = 1 mod 2N: an element
// of multiplicative order 2N (N a power of two) is exactly one with x^N = -1.
// A quadratic non-residue g gives h = g^((q-1)/2N) with h^N = -1; the 2N-th
// primitive roots are then the odd powers of h.
uint64_t min_primitive_root(uint64_t N, uint64_t q) {
    uint64_t h = 0;
    for (uint64_t g = 2; g < q && g < (1ull << 24); ++g) {
        uint64_t c = powmod_u64(g, (q - 1) / (2 * N), q);
        if (powmod_u64(c, N, q) == q - 1) { h = c; break; }
    }
    if (!h) return 0;
    uint64_t h2 = mulmod(h, h, q), x = h, best = h;
    for (uint64_t k = 1; k < N; ++k) {
        x = mulmod(x, h2, q);
        best = std::min(best, x);
    }
    return best;
}

// Smallest primitive N-th root of unity mod prime q = 1 mod N (N a power of
// two >= 2): x has order N exactly when x^(N/2) = -1; h = g^((q-1)/N) for a
// quadratic non-residue g has that property, and the primitive N-th roots are
// the odd powers of h.
uint64_t min_primitive_nth_root(uint64_t N, uint64_t q) {
    uint64_t h = 0;
    for (uint64_t g = 2; g < q && g < (1ull << 24); ++g) {
        uint64_t c = powmod_u64(g, (q - 1) / N, q);
        if (powmod_u64(c, N / 2, q) == q - 1) { h = c; break; }
    }
    if (!h) return 0;
    uint64_t h2 = mulmod(h, h, q), x = h, best = h;
    for (uint64_t k = 1; k < N / 2; ++k) {
        x = mulmod(x, h2, q);
        best = std::min(best, x);
    }
    return best;
}

static inline uint64_t bitrev(uint64_t i, int logn) {
    uint64_t r = 0;
    for (int b = 0; b < logn; ++b) { r = (r << 1) | (i & 1); i >>= 1; }
    return r;
}

static inline uint64_t shoup(uint64_t w, uint64_t q, bool narrow) {
    return narrow ? (uint64_t)(((uint64_t)w << 32) / q) : (uint64_t)(((u128)w << 64) / q);
}

// Fill one limb's tables (host staging buffers of N pairs each); `root` is
// psi (negacyclic) or omega (cyclic).
static void fill_limb(uint64_t N, int logN, uint64_t q, uint64_t root, bool cyclic,
                      ulonglong2* fwd, ulonglong2* inv, LimbDev* ld) {
    const bool narrow = q < (1ull << 30);
    const uint64_t root_inv = powmod_u64(root, q - 2, q);
    std::vector<uint64_t> pw(N), pwi(N);
    pw[0] = pwi[0] = 1;
    for (uint64_t i = 1; i < N; ++i) {
        pw[i] = mulmod(pw[i - 1], root, q);
        pwi[i] = mulmod(pwi[i - 1], root_inv, q);
    }
    for (uint64_t k = 0; k < N; ++k) {
        uint64_t r;
        if (!cyclic) {
            r = bitrev(k, logN);
        } else {
            int sb = 0;
            while (k >> (sb + 1)) ++sb;   // k = 2^sb + i
            r = k ? bitrev(k - (1ull << sb), sb) << (logN - 1 - sb) : 0;
        }
        uint64_t w = k ? pw[r] : 1, wi = k ? pwi[r] : 1;
        fwd[k] = make_ulonglong2(w, shoup(w, q, narrow));
        inv[k] = make_ulonglong2(wi, shoup(wi, q, narrow));
    }
    uint64_t ninv = powmod_u64(N % q, q - 2, q);
    uint64_t ninv_w = mulmod(ninv, inv[1].x, q);
    ld->q = q;
    ld->two_q = 2 * q;
    ld->ninv = ninv;
    ld->ninv_p = shoup(ninv, q, narrow);
    ld->ninv_w = ninv_w;
    ld->ninv_w_p = shoup(ninv_w, q, narrow);
    ld->narrow = narrow ? 1u : 0u;
    ld->trunc = (!narrow && q < (1ull << 61)) ? 1u : 0u;
    ld->pad_ = 0;
    int Q = 0;
    while (Q < 64 && (q >> Q)) ++Q;   // bit length; q is an odd prime, so q > 2^(Q-1)
    ld->barrett_qm1 = (uint32_t)(Q - 1);
    ld->barrett_k = (uint64_t)(((u128)1 << (63 + Q)) / q);
}

// Untuned default schedules (the autotuner replaces them per workload).  For
// N > 2^13: a column pass over the first log2(N)/2 stages in 8- or 4-column
// tiles, then a row pass over the rest in small row tiles of 8 elements a
// thread -- the fastest shapes of a sweep at N = 2^16 on 32 mixed limbs.
NttCfg default_cfg(int logN, bool forward) {
    NttCfg c{};
    if (logN <= 13) {
        c.npass = 1;
        c.pass[0] = PassCfg{0, logN, 0, 0, logN <= 12 ? 3 : 4, 0, 1};
    } else {
        const int K1 = logN / 2, K2 = logN - K1;
        c.npass = 2;
        c.pass[0] = forward ? PassCfg{0, K1, 0, 3, 4, 0, 1} : PassCfg{0, K1, 0, 2, 3, 0, 1};
        const int logGb = std::max(forward ? 0 : 1, 8 - K2);
        c.pass[1] = PassCfg{K1, K2, std::min(logGb, K1), 0, 3, 0, 1};
    }
    return c;
}

// ---------------------------------------------------------------- table cache
// Twiddle tables depend only on (device, N, q, psi), so plans share them: a
// process-wide map holds weak references, plans hold strong ones, and a table
// is freed with the last plan that uses it.  Many plans over overlapping
// prime sets (ragged batches, served requests) then cost one table per
// distinct (N, q, psi).
TableEntry::~TableEntry() {
    if (!d_mem) return;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != device) cudaSetDevice(device);
    cudaFree(d_mem);
    if (prev != device) cudaSetDevice(prev);
}

namespace {
typedef std::tuple<int, uint64_t, uint64_t, uint64_t> TableKey;
std::mutex g_table_mu;
std::map<TableKey, std::weak_ptr<TableEntry>> g_tables;
}  // namespace

// (device, N, q, root) identifies a table: a cyclic plan's omega has order N,
// a negacyclic plan's psi order 2N, so the two kinds never share a key.
int acquire_tables(int device, uint64_t N, int logN, const std::vector<uint64_t>& moduli,
                   const std::vector<uint64_t>& roots, bool cyclic,
                   std::vector<std::shared_ptr<TableEntry>>* out) {
    std::lock_guard<std::mutex> g(g_table_mu);
    const size_t L = moduli.size();
    out->assign(L, nullptr);
    std::vector<size_t> missing;
    std::map<TableKey, size_t> first_of;   // duplicates within one plan share one fill
    for (size_t l = 0; l < L; ++l) {
        const TableKey key(device, N, moduli[l], roots[l]);
        auto it = g_tables.find(key);
        if (it != g_tables.end()) (*out)[l] = it->second.lock();
        if (!(*out)[l] && !first_of.count(key)) {
            first_of[key] = l;
            missing.push_back(l);
        }
    }
    // fill the new tables on the host in parallel, then upload each
    std::vector<std::vector<ulonglong2>> host(missing.size());
    std::vector<LimbDev> lds(missing.size());
    unsigned nthreads = std::max(1u, std::min(std::thread::hardware_concurrency(), 16u));
    nthreads = std::min<unsigned>(nthreads, (unsigned)std::max<size_t>(missing.size(), 1));
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nthreads; ++t) {
        pool.emplace_back([&, t]() {
            for (size_t m = t; m < missing.size(); m += nthreads) {
                const size_t l = missing[m];
                host[m].resize(2 * N);
                fill_limb(N, logN, moduli[l], roots[l], cyclic, host[m].data(),
                          host[m].data() + N, &lds[m]);
            }
        });
    }
    for (auto& th : pool) th.join();
    for (size_t m = 0; m < missing.size(); ++m) {
        const size_t l = missing[m];
        auto e = std::make_shared<TableEntry>();
        e->device = device;
        e->bytes = 2 * N * sizeof(ulonglong2);
        if (cudaMalloc(&e->d_mem, e->bytes) != cudaSuccess) {
            e->d_mem = nullptr;
            out->clear();
            return HX_ERR_NOMEM;
        }
        if (cudaMemcpy(e->d_mem, host[m].data(), e->bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
            out->clear();
            return HX_ERR_CUDA;
        }
        e->ld = lds[m];
        e->ld.fwd = (const ulonglong2*)e->d_mem;
        e->ld.inv = (const ulonglong2*)e->d_mem + N;
        const TableKey key(device, N, moduli[l], roots[l]);
        g_tables[key] = e;
        (*out)[l] = e;
    }
    for (size_t l = 0; l < L; ++l) {
        if (!(*out)[l]) (*out)[l] = g_tables[TableKey(device, N, moduli[l], roots[l])].lock();
    }
    // forget expired entries
    for (auto it = g_tables.begin(); it != g_tables.end();) {
        if (it->second.expired())
            it = g_tables.erase(it);
        else
            ++it;
    }
    return HX_OK;
}

// The launch order of a plan's limbs (see hx_plan_s::d_order): within each
// run of 64, limbs by decreasing cost of their butterfly, ties in index order.
std::vector<uint32_t> launch_order(const std::vector<LimbDev>& limbs) {
    auto cost = [&](uint32_t l) { return limbs[l].narrow ? 0 : limbs[l].trunc ? 1 : 2; };
    const uint32_t n = (uint32_t)limbs.size();
    std::vector<uint32_t> order(n);
    for (uint32_t l = 0; l < n; ++l) order[l] = l;
    for (uint32_t b = 0; b < n; b += 64)
        std::stable_sort(order.begin() + b, order.begin() + std::min(n, b + 64),
                         [&](uint32_t x, uint32_t y) { return cost(x) > cost(y); });
    return order;
}

}  // namespace hx

using namespace hx;

// Plan creation for both kinds: negacyclic (roots psi of order 2N, q = 1
// mod 2N) and cyclic (roots omega of order N, q = 1 mod N).
static int plan_create(hx_plan_t* out, uint64_t N, const uint64_t* h_moduli, uint32_t n_limbs,
                       const uint64_t* h_roots, bool cyclic) {
    if (!out || !h_moduli) return HX_ERR_NULL;
    *out = nullptr;
    if (N < 1024 || N > (1u << 17) || (N & (N - 1))) return HX_ERR_DEGREE;
    if (n_limbs == 0 || n_limbs > 4096) return HX_ERR_ARG;
    int logN = 0;
    while ((1ull << logN) < N) ++logN;
    const uint64_t order = cyclic ? N : 2 * N;   // order of the root
    std::vector<uint64_t> roots(n_limbs);
    for (uint32_t l = 0; l < n_limbs; ++l) {
        uint64_t q = h_moduli[l];
        if (q < 3 || q >= (1ull << 62) || (q - 1) % order != 0 || !is_prime_u64(q))
            return HX_ERR_MODULUS;
        if (h_roots) {
            uint64_t r = h_roots[l];
            if (r == 0 || r >= q || powmod_u64(r, order / 2, q) != q - 1) return HX_ERR_ROOT;
            roots[l] = r;
        } else {
            roots[l] = cyclic ? min_primitive_nth_root(N, q) : min_primitive_root(N, q);
            if (!roots[l]) return HX_ERR_MODULUS;
        }
    }
    hx_plan_s* p = new (std::nothrow) hx_plan_s();
    if (!p) return HX_ERR_NOMEM;
    p->N = N;
    p->logN = logN;
    p->n_limbs = n_limbs;
    p->cyclic = cyclic;
    p->moduli.assign(h_moduli, h_moduli + n_limbs);
    p->roots = roots;
    p->cfg_fwd = default_cfg(logN, true);
    p->cfg_inv = default_cfg(logN, false);
    cudaGetDevice(&p->device);
    int st = acquire_tables(p->device, N, logN, p->moduli, roots, cyclic, &p->tables);
    if (st != HX_OK) {
        delete p;
        return st;
    }
    p->h_limbs.resize(n_limbs);
    for (uint32_t l = 0; l < n_limbs; ++l) p->h_limbs[l] = p->tables[l]->ld;
    p->h_order = launch_order(p->h_limbs);
    const size_t limb_bytes = n_limbs * sizeof(LimbDev);
    const size_t bytes = limb_bytes + n_limbs * sizeof(uint32_t);
    if (cudaMalloc((void**)&p->d_limbs, bytes) != cudaSuccess) {
        delete p;
        return HX_ERR_NOMEM;
    }
    p->d_order = reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(p->d_limbs) + limb_bytes);
    if (cudaMemcpy(p->d_limbs, p->h_limbs.data(), limb_bytes, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(p->d_order, p->h_order.data(), n_limbs * sizeof(uint32_t),
                   cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(p->d_limbs);
        delete p;
        return HX_ERR_CUDA;
    }
    p->device_bytes = bytes;
    std::vector<const TableEntry*> seen;
    for (auto& t : p->tables) {
        if (std::find(seen.begin(), seen.end(), t.get()) == seen.end()) {
            seen.push_back(t.get());
            p->device_bytes += t->bytes;
        }
    }
    *out = p;
    return HX_OK;
}

extern "C" int hx_plan_create(hx_plan_t* out, uint64_t N, const uint64_t* h_moduli,
                              uint32_t n_limbs, const uint64_t* h_roots) {
    return plan_create(out, N, h_moduli, n_limbs, h_roots, false);
}

extern "C" int hx_plan_create_cyclic(hx_plan_t* out, uint64_t N, const uint64_t* h_moduli,
                                     uint32_t n_limbs, const uint64_t* h_roots) {
    return plan_create(out, N, h_moduli, n_limbs, h_roots, true);
}

extern "C" int hx_plan_destroy(hx_plan_t p) {
    if (!p) return HX_ERR_NULL;
    int prev = 0;
    cudaGetDevice(&prev);
    if (prev != p->device) cudaSetDevice(p->device);
    cudaFree(p->d_limbs);
    p->tables.clear();   // drops this plan's references; unused tables are freed
    if (prev != p->device) cudaSetDevice(prev);
    delete p;
    return HX_OK;
}

extern "C" int hx_plan_roots(hx_plan_t p, uint64_t* h_roots_out) {
    if (!p || !h_roots_out) return HX_ERR_NULL;
    memcpy(h_roots_out, p->roots.data(), p->n_limbs * sizeof(uint64_t));
    return HX_OK;
}

extern "C" int hx_plan_info(hx_plan_t p, uint64_t* N, uint32_t* n_limbs, uint64_t* bytes) {
    if (!p) return HX_ERR_NULL;
    if (N) *N = p->N;
    if (n_limbs) *n_limbs = p->n_limbs;
    if (bytes) *bytes = p->device_bytes;
    return HX_OK;
}

extern "C" int hx_plan_set_schedule(hx_plan_t p, uint32_t direction, uint32_t npass,
                                    const int32_t* params) {
    if (!p || !params) return HX_ERR_NULL;
    if (npass < 1 || npass > 2 || direction < 1 || direction > 3) return HX_ERR_ARG;
    NttCfg c{};
    c.npass = (int)npass;
    for (uint32_t i = 0; i < npass; ++i) {
        const int32_t* q = params + 7 * i;
        c.pass[i] = PassCfg{q[0], q[1], q[2], q[3], q[4], q[5], q[6]};
    }
    if (!cfg_supported(p->logN, c)) return HX_ERR_ARG;
    if (direction & 1) p->cfg_fwd = c;
    if (direction & 2) p->cfg_inv = c;
    return HX_OK;
}

extern "C" int hx_plan_get_schedule(hx_plan_t p, uint32_t direction, uint32_t* npass,
                                    int32_t* params) {
    if (!p || !npass || !params) return HX_ERR_NULL;
    if (direction != 1 && direction != 2) return HX_ERR_ARG;
    const NttCfg& cfg = direction == 1 ? p->cfg_fwd : p->cfg_inv;
    *npass = (uint32_t)cfg.npass;
    for (int i = 0; i < 2; ++i) {
        const PassCfg& c = cfg.pass[i];
        const int32_t v[7] = {c.s0, c.K, c.logGb, c.logGc, c.logR, c.pipe, c.np};
        memcpy(params + 7 * i, v, sizeof(v));
    }
    return HX_OK;
}
