// Grouped GEMM: many independent C_g = alpha_g op(A_g) op(B_g) + beta_g C_g
// in one split launch plus one persistent tensor-core launch.
//
// Not in the paper.  Its per-target blocking parameters (mc, kc, nc chosen
// from cache sizes, Section 3.1, Eqs. 1-7) have a GPU analogue here: the
// tile width BN, the stage depth BK and the ring depth are chosen per launch
// by an autotuner whose analytic seed is a feasibility-and-cost model of
// shared memory (227 KB per CTA), tensor memory (512 columns per SM) and
// tile quantisation, refined by timing the surviving candidates on the
// problems themselves.
//
// A plan owns its device tables (problem descriptors, tensor maps, split
// jobs) and the BF16 hi/lo workspace; running it enqueues only kernels, so
// it can be captured into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gemm.h"
#include "internal.h"

struct gemm_grouped_plan_s {
    gemm_handle_t handle = nullptr;
    int device = 0;
    int num_sms = 0;
    int* err_word = nullptr;
    int nterms = 3;
    uint32_t flags = 0;
    gb300::TcLaunch cfg;
    double tuned_ms = 0.0;
    // device allocations owned by the plan
    uint8_t* ws = nullptr;
    gb300::SplitJob* d_jobs = nullptr;
    gb300::GroupedProblem* d_probs = nullptr;
    CUtensorMap* d_maps = nullptr;
    int* d_tile_prob = nullptr;
    int* d_tile_job = nullptr;    // tiles of direct (non-transposed) jobs
    int* d_tile_job_t = nullptr;  // tiles of transposed jobs
    int split_tiles_t = 0;
    int njobs = 0, split_tiles = 0, nprobs = 0, total_tiles = 0;
    // problems handled by a plain scale (K == 0 or alpha == 0)
    struct Scale {
        int64_t M, N, ldc;
        float beta;
        float* C;
    };
    std::vector<Scale> scales;
    // per-problem split-K: the slices' partial sums (plan-owned) and the
    // reduces that add them into the callers' C after the grouped launch
    float* partials = nullptr;
    struct KReduce {
        int64_t M, N, ldc;
        int split;
        float* P;
        float alpha, beta;
        float* C;
    };
    std::vector<KReduce> reduces;
    gb300::ReduceJob* d_reduces = nullptr;  // their device table: one reduce launch
    long long reduce_units = 0;
    int max_split = 1;
    // graph replay
    cudaGraphExec_t exec = nullptr;
    cudaStream_t exec_stream = nullptr;
    int launches = 0;
};

namespace {

using gb300::GroupedProblem;
using gb300::SplitJob;
using gb300::TcLaunch;
using gb300::TcOperand;

size_t round256(size_t x) { return (x + 255) / 256 * 256; }

// One tensor-core problem of the plan, host side.
struct HostProb {
    TcOperand a, b;
    int64_t M, N, K, ldc;
    float alpha, beta;
    float* C;
};

// Problem table and tensor maps for a tile shape; returns total tiles.
// Tiles are 128 x bn (one CTA) or 256 x bn (CTA pairs, each CTA staging
// bn / 2 rows of B).
int build_tables(const std::vector<HostProb>& ps, const TcLaunch& cfg,
                 std::vector<GroupedProblem>& probs, std::vector<CUtensorMap>& maps,
                 std::vector<int>& tile_prob, bool* ok) {
    const int bn = cfg.bn, bk = cfg.bk;
    const int cg = cfg.cta_group == 2 ? 2 : 1;
    probs.clear();
    tile_prob.clear();
    maps.assign(2 * ps.size(), CUtensorMap{});
    int tiles = 0;
    *ok = true;
    for (size_t i = 0; i < ps.size(); ++i) {
        const HostProb& q = ps[i];
        GroupedProblem g{};
        g.C = q.C;
        g.ldc = q.ldc;
        g.M = int(q.M);
        g.N = int(q.N);
        g.K = int(q.K);
        g.num_m = int((q.M + 128 * cg - 1) / (128 * cg));
        g.num_n = int((q.N + bn - 1) / bn);
        g.k_blocks = int((q.K + bk - 1) / bk);
        g.tile_start = tiles;
        g.alpha = q.alpha;
        g.beta = q.beta;
        g.major = (q.a.mn_major ? 1 : 0) | (q.b.mn_major ? 2 : 0);
        tiles += g.num_m * g.num_n;
        tile_prob.insert(tile_prob.end(), size_t(g.num_m) * g.num_n, int(i));
        probs.push_back(g);
        if (!gb300::encode_operand(&maps[2 * i], q.a, bk, 128) ||
            !gb300::encode_operand(&maps[2 * i + 1], q.b, bk, bn / cg))
            *ok = false;
    }
    return tiles;
}

// Analytic seed: which (BN, BK, one CTA or CTA pairs) exist on this SM and
// what they should cost.  Cost = padded tensor work of every tile (tiles are
// 128 x BN or, for pairs, 256 x BN, and K is padded to BK, so ragged edges
// waste work) times the wave-quantisation factor of the persistent grid,
// divided by the configuration's efficiency: its padded work per second,
// measured on 512 uneven problems (M, N, K in 32 * U{2..64}, 3xBF16) with the
// split pass subtracted, relative to the fastest.  Pairs with BK 64 ran at
// the sustained tensor rate; smaller stages pay a per-stage issue cost that
// no padding term shows (one CTA with BN 128 and BK 32 at 0.68), and one CTA
// per tile stays below pairs per clock (0.90 with BN 256, BK 32).
// The in-kernel split (one CTA, BN 256, BK 32, `fused`) pays for its
// converter warps with a lower rate than the same tiles on pre-split
// operands, but needs no split pass.
double config_efficiency(int cg, int bn, int bk, bool fused = false) {
    if (fused) return 0.55;
    if (cg == 2) return bk == 64 ? 1.00 : 0.91;
    if (bn == 256) return bk == 32 ? 0.90 : 0.83;
    return bk == 64 ? 0.80 : 0.68;
}

struct Candidate {
    TcLaunch cfg;
    double model;  // seconds: kernel estimate, plus the split pass when it needs one
};

// Estimated seconds of the split pass over every operand: 8 bytes of HBM
// traffic per element of A and B at about 5.8 TB/s.
double split_pass_seconds(const std::vector<HostProb>& ps) {
    double elems = 0.0;
    for (const HostProb& q : ps) elems += double(q.M) * q.K + double(q.N) * q.K;
    return 8.0 * elems / 5.8e12;
}

// Candidate configurations ranked by the model.  `prepass` / `fused` say
// which split placements may be considered.
std::vector<Candidate> seed_candidates(const std::vector<HostProb>& ps, int nterms, int num_sms,
                                       const TcLaunch& base, bool prepass = true,
                                       bool fused = false) {
    std::vector<Candidate> out;
    const int kmax_smem = 232448;
    const double t_split = split_pass_seconds(ps);
    const double flop_per_mac = 2.0 * nterms;
    for (int f : {0, 1}) {
    if ((f == 0 && !prepass) || (f == 1 && (!fused || nterms != 3))) continue;
    for (int cg : {1, 2}) {
        for (int bn : {256, 128}) {
            for (int bk : {32, 64}) {
                if (f == 1 && (cg != 1 || bn != 256 || bk != 32)) continue;  // fused shape
                if (cg == 2 && (bn != 256 || nterms != 3)) continue;  // pair kernels compiled
                int stages = 0;
                for (int s = 8; s >= 2; --s)
                    if (gb300::tc_smem_bytes(nterms, bn, bk, s, cg) <= kmax_smem) {
                        stages = s;
                        break;
                    }
                if (stages < 2 || 2 * bn > 512) continue;  // shared memory or TMEM does not fit
                const int bm = 128 * cg;
                double work = 0.0, tiles = 0.0;
                for (const HostProb& q : ps) {
                    const double nm = double((q.M + bm - 1) / bm), nn = double((q.N + bn - 1) / bn);
                    const double kk = double((q.K + bk - 1) / bk) * bk;
                    work += nm * nn * double(bm) * bn * kk;
                    tiles += nm * nn;
                }
                const double units = double(num_sms / cg);  // CTAs or CTA pairs
                const double waves = std::ceil(tiles / units) / (tiles / units);
                Candidate c;
                c.cfg = base;
                c.cfg.bn = bn;
                c.cfg.bk = bk;
                c.cfg.stages = stages;
                c.cfg.split_k = 1;
                c.cfg.cta_group = cg;
                c.cfg.fuse = f ? 3 : 0;  // both operands split in the kernel
                c.cfg.kmajor = f ? 0 : base.kmajor;
                c.model = flop_per_mac * work * waves / (1.8e15 * config_efficiency(cg, bn, bk, f)) +
                          (f ? 0.0 : t_split);
                out.push_back(c);
            }
        }
    }
    }
    std::sort(out.begin(), out.end(),
              [](const Candidate& x, const Candidate& y) { return x.model < y.model; });
    return out;
}

// Per-problem split-K (a grouped analogue of gemm()'s split-K for few-tile,
// long-K problems): under a tile configuration, a problem whose one tile
// carries more K blocks than a CTA's (or CTA pair's) even share of the whole
// launch would finish last.  It is cut into S slices (up to 8, at least 4 K
// blocks each); slice j is a problem of its own over K blocks [j per, (j+1)
// per) that stores its raw partial sum (alpha 1, beta 0) in slab j of a
// plan-owned buffer, and a reduce launch adds the slabs in slice order into C
// with alpha and beta, as gemm()'s split-K does.  Returns S per problem.
std::vector<int> straggler_splits(const std::vector<HostProb>& ps, const TcLaunch& cfg,
                                  int num_sms) {
    const int cg = cfg.cta_group == 2 ? 2 : 1;
    const int bm = 128 * cg, bn = cfg.bn, bk = cfg.bk;
    double units = 0.0;
    for (const HostProb& q : ps)
        units += double((q.M + bm - 1) / bm) * double((q.N + bn - 1) / bn) *
                 double((q.K + bk - 1) / bk);
    const double share = std::max(4.0, units / double(std::max(1, num_sms / cg)));
    std::vector<int> out;
    for (const HostProb& q : ps) {
        const int64_t kb = (q.K + bk - 1) / bk;
        int64_t sp = 1;
        if (double(kb) > share) sp = std::min<int64_t>({8, int64_t(std::ceil(kb / share)), kb / 4});
        out.push_back(int(std::max<int64_t>(sp, 1)));
    }
    return out;
}

// Slice [k0, k0 + k) of an operand's K range (a view of the same planes).
TcOperand k_slice(const TcOperand& op, int64_t k0, int64_t k) {
    TcOperand t = op;
    t.base = op.base + (op.mn_major ? k0 * op.ld : k0);
    t.k = k;
    return t;
}

// The problems with every split problem replaced by its slices (their C the
// partial slabs at `partials`, laid out problem by problem in order), and
// the reduces that finish them.  Returns the float count of the slabs.
size_t slice_problems(const std::vector<HostProb>& ps, const std::vector<int>& splits, int bk,
                      float* partials, std::vector<HostProb>* out,
                      std::vector<gemm_grouped_plan_s::KReduce>* reduces) {
    out->clear();
    if (reduces) reduces->clear();
    size_t off = 0;
    for (size_t i = 0; i < ps.size(); ++i) {
        const HostProb& q = ps[i];
        const int sp = splits.empty() ? 1 : splits[i];
        if (sp <= 1) {
            out->push_back(q);
            continue;
        }
        const int64_t kb = (q.K + bk - 1) / bk;
        const int64_t per = (kb + sp - 1) / sp;
        const int slices = int((kb + per - 1) / per);
        float* P = partials ? partials + off : nullptr;
        for (int j = 0; j < slices; ++j) {
            const int64_t k0 = j * per * bk, k1 = std::min<int64_t>(q.K, (j + 1) * per * bk);
            HostProb sq = q;
            sq.a = k_slice(q.a, k0, k1 - k0);
            sq.b = k_slice(q.b, k0, k1 - k0);
            sq.K = k1 - k0;
            sq.C = P ? P + size_t(j) * size_t(q.M) * size_t(q.N) : nullptr;
            sq.ldc = q.N;
            sq.alpha = 1.0f;
            sq.beta = 0.0f;
            out->push_back(sq);
        }
        if (reduces) reduces->push_back({q.M, q.N, q.ldc, slices, P, q.alpha, q.beta, q.C});
        off += size_t(slices) * size_t(q.M) * size_t(q.N);
    }
    return off;
}

// The reduces as one launch's job table; returns the total units.
long long reduce_table(const std::vector<gemm_grouped_plan_s::KReduce>& reds,
                       std::vector<gb300::ReduceJob>* jobs) {
    jobs->clear();
    long long units = 0;
    for (const auto& r : reds) {
        gb300::ReduceJob j{};
        j.P = r.P;
        j.C = r.C;
        j.M = r.M;
        j.N = r.N;
        j.ldc = r.ldc;
        j.split = r.split;
        j.alpha = r.alpha;
        j.beta = r.beta;
        j.vec = (r.N % 4 == 0) && (r.ldc % 4 == 0) &&
                ((reinterpret_cast<uintptr_t>(r.C) & 15) == 0) &&
                ((reinterpret_cast<uintptr_t>(r.P) & 15) == 0);
        j.unit_start = units;
        units += j.vec ? r.M * r.N / 4 : r.M * r.N;
        jobs->push_back(j);
    }
    return units;
}

std::string shape_key(int device_sms, int nterms, const std::vector<HostProb>& ps) {
    // order-independent signature: count and a hash of the sorted shapes
    std::vector<uint64_t> v;
    for (const HostProb& q : ps)
        v.push_back((uint64_t(q.M) << 42) ^ (uint64_t(q.N) << 21) ^ uint64_t(q.K) ^
                    (uint64_t(q.a.mn_major + 2 * q.b.mn_major) << 62));
    std::sort(v.begin(), v.end());
    uint64_t h = 1469598103934665603ull;
    for (uint64_t x : v) {
        h ^= x;
        h *= 1099511628211ull;
    }
    char buf[96];
    snprintf(buf, sizeof buf, "sms%d-t%d-n%zu-%016llx", device_sms, nterms, ps.size(),
             (unsigned long long)h);
    return buf;
}

std::mutex g_cache_mu;
std::map<std::string, TcLaunch> g_cache;

bool cache_lookup(const std::string& key, TcLaunch* out) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) {
        *out = it->second;
        return true;
    }
    // optional persistent cache: lines "key bn bk stages raster cta_group fuse
    // ksplit" (a missing cta_group means one CTA, a missing fuse the split
    // pass, a missing ksplit no per-problem split-K)
    const char* path = getenv("GEMM_AUTOTUNE_CACHE");
    if (!path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[256], k[128];
    bool found = false;
    while (fgets(line, sizeof line, f)) {
        int bn, bk, st, rg, cg = 1, fu = 0, ks = 0;
        const int n =
            sscanf(line, "%127s %d %d %d %d %d %d %d", k, &bn, &bk, &st, &rg, &cg, &fu, &ks);
        if (n < 5 || key != k) continue;
        out->bn = bn;
        out->bk = bk;
        out->stages = st;
        out->raster_group = rg;
        out->cta_group = cg == 2 ? 2 : 1;
        out->fuse = fu == 1 ? 3 : 0;
        out->split_k = ks == 1 ? 2 : 1;  // 2: split stragglers
        found = true;
    }
    fclose(f);
    if (found) g_cache[key] = *out;
    return found;
}

void cache_store(const std::string& key, const TcLaunch& c) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_cache[key] = c;
    const char* path = getenv("GEMM_AUTOTUNE_CACHE");
    if (!path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s %d %d %d %d %d %d %d\n", key.c_str(), c.bn, c.bk, c.stages, c.raster_group,
            c.cta_group, c.fuse ? 1 : 0, c.split_k > 1 ? 1 : 0);
    fclose(f);
}

template <typename T>
gemm_status_t upload(T** dst, const std::vector<T>& v, cudaStream_t s) {
    if (v.empty()) return GEMM_OK;
    if (!*dst && cudaMalloc(reinterpret_cast<void**>(dst), v.size() * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        return GEMM_ERR_WORKSPACE;
    }
    if (cudaMemcpyAsync(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return GEMM_ERR_CUDA;
    return GEMM_OK;
}

void free_plan(gemm_grouped_plan_s* p) {
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->ws) cudaFree(p->ws);
    if (p->partials) cudaFree(p->partials);
    if (p->d_reduces) cudaFree(p->d_reduces);
    if (p->d_jobs) cudaFree(p->d_jobs);
    if (p->d_probs) cudaFree(p->d_probs);
    if (p->d_maps) cudaFree(p->d_maps);
    if (p->d_tile_prob) cudaFree(p->d_tile_prob);
    if (p->d_tile_job) cudaFree(p->d_tile_job);
    if (p->d_tile_job_t) cudaFree(p->d_tile_job_t);
    delete p;
}

// Time one configuration on (a subset of) the problems with C redirected to
// plan-owned scratch and beta = 0, so the caller's C is never touched; with
// `reds`, the split-K reduces after the grouped launch are timed too.
double time_candidate(const std::vector<HostProb>& sub, int nterms, const TcLaunch& cfg,
                      int* err_word, int num_sms, cudaStream_t s,
                      const std::vector<gemm_grouped_plan_s::KReduce>* reds = nullptr) {
    std::vector<gb300::ReduceJob> rjobs;
    const long long runits = reds ? reduce_table(*reds, &rjobs) : 0;
    gb300::ReduceJob* dr = nullptr;
    std::vector<GroupedProblem> probs;
    std::vector<CUtensorMap> maps;
    std::vector<int> tile_prob;
    bool ok = true;
    const int tiles = build_tables(sub, cfg, probs, maps, tile_prob, &ok);
    if (!ok) return -1.0;
    GroupedProblem* dp = nullptr;
    CUtensorMap* dm = nullptr;
    int* dt = nullptr;
    double best = -1.0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (upload(&dp, probs, s) == GEMM_OK && upload(&dm, maps, s) == GEMM_OK &&
        upload(&dt, tile_prob, s) == GEMM_OK && upload(&dr, rjobs, s) == GEMM_OK &&
        cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
        for (int rep = 0; rep < 4; ++rep) {
            cudaEventRecord(e0, s);
            int rc = gb300::launch_tc_grouped(nterms, cfg, dp, dm, dt, int(sub.size()), tiles,
                                              err_word, num_sms, s);
            if (rc == 0 && !rjobs.empty() &&
                gb300::launch_splitk_reduce_grouped(dr, int(rjobs.size()), runits, num_sms, s) !=
                    cudaSuccess)
                rc = -4;
            cudaEventRecord(e1, s);
            if (rc != 0 || cudaEventSynchronize(e1) != cudaSuccess) {
                best = -1.0;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (best < 0.0 || ms < best)) best = ms;  // first launch is warm-up
        }
    }
    cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (dp) cudaFree(dp);
    if (dm) cudaFree(dm);
    if (dt) cudaFree(dt);
    if (dr) cudaFree(dr);
    return best;
}

// The same configuration with the straggler problems split along K (their
// slices' partial sums in a temporary buffer, the reduces writing the
// subset's scratch C); a negative time when there is nothing to split or no
// memory.
double time_split_variant(const std::vector<HostProb>& sub, int nterms, const TcLaunch& cfg,
                          int* err_word, int num_sms, cudaStream_t s) {
    const std::vector<int> splits = straggler_splits(sub, cfg, num_sms);
    if (*std::max_element(splits.begin(), splits.end()) <= 1) return -1.0;
    std::vector<HostProb> sliced;
    const size_t floats = slice_problems(sub, splits, cfg.bk, nullptr, &sliced, nullptr);
    float* buf = nullptr;
    if (cudaMalloc(reinterpret_cast<void**>(&buf), floats * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return -1.0;
    }
    std::vector<gemm_grouped_plan_s::KReduce> reds;
    slice_problems(sub, splits, cfg.bk, buf, &sliced, &reds);
    const double ms = time_candidate(sliced, nterms, cfg, err_word, num_sms, s, &reds);
    cudaFree(buf);
    return ms;
}

gemm_status_t enqueue(gemm_grouped_plan_s* p, cudaStream_t s) {
    for (const auto& sc : p->scales)
        if (gb300::launch_scale_c(sc.M, sc.N, sc.beta, sc.C, sc.ldc, s) != cudaSuccess)
            return GEMM_ERR_CUDA;
    if (gb300::launch_split_grouped(p->d_jobs, p->d_tile_job, p->njobs, p->split_tiles,
                                    p->num_sms, s) != cudaSuccess ||
        gb300::launch_split_grouped_t(p->d_jobs, p->d_tile_job_t, p->njobs, p->split_tiles_t,
                                      p->num_sms, s) != cudaSuccess)
        return GEMM_ERR_CUDA;
    const int rc = gb300::launch_tc_grouped(p->nterms, p->cfg, p->d_probs, p->d_maps,
                                            p->d_tile_prob, p->nprobs, p->total_tiles,
                                            p->err_word, p->num_sms, s);
    if (rc != 0) return static_cast<gemm_status_t>(rc);
    if (p->d_reduces && gb300::launch_splitk_reduce_grouped(p->d_reduces, int(p->reduces.size()),
                                                            p->reduce_units, p->num_sms,
                                                            s) != cudaSuccess)
        return GEMM_ERR_CUDA;
    return GEMM_OK;
}

}  // namespace

// Declared by api.cu's context; grouped.cu only needs these three fields.
namespace gb300 {
int handle_device(gemm_handle_t h);
int handle_num_sms(gemm_handle_t h);
int* handle_err_word(gemm_handle_t h);
void handle_set_err_arg(gemm_handle_t h, int pos);
void handle_set_launches(gemm_handle_t h, int n);
TcLaunch handle_tc_config(gemm_handle_t h, int nterms);
bool handle_tile_auto(gemm_handle_t h);
int handle_split_place(gemm_handle_t h);
int handle_split_k(gemm_handle_t h);
}  // namespace gb300

extern "C" {

gemm_status_t gemm_grouped_plan_create(gemm_handle_t h, gemm_mode_t mode,
                                       const gemm_problem_t* hp, int32_t count, uint32_t flags,
                                       void* stream, gemm_grouped_plan_t* plan) {
    if (!h) return GEMM_ERR_ARG;
    gb300::handle_set_err_arg(h, 0);
    auto bad = [&](int pos) {
        gb300::handle_set_err_arg(h, pos);
        return GEMM_ERR_ARG;
    };
    if (mode != GEMM_MODE_BF16 && mode != GEMM_MODE_BF16X3) return bad(2);
    // one placement for both operands of every problem (no per-operand choice)
    if (gb300::handle_split_place(h) > GEMM_SPLIT_IN_KERNEL) return bad(1);
    if (count < 0) return bad(4);
    if (count > 0 && !hp) return bad(3);
    if (flags & ~uint32_t(GEMM_GROUPED_AUTOTUNE | GEMM_GROUPED_GRAPH)) return bad(5);
    if (!plan) return bad(7);
    *plan = nullptr;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nterms = mode == GEMM_MODE_BF16X3 ? 3 : 1;
    const int planes = nterms == 3 ? 2 : 1;

    // validate every problem exactly as gemm() would
    for (int i = 0; i < count; ++i) {
        const gemm_problem_t& q = hp[i];
        const bool ta = q.transA != 0, tb = q.transB != 0;
        const bool reads = q.M > 0 && q.N > 0 && q.K > 0 && q.alpha != 0.0f;
        const int64_t lim = (int64_t(1) << 31) - 1024;
        if ((q.transA != 0 && q.transA != 1) || (q.transB != 0 && q.transB != 1) || q.M < 0 ||
            q.N < 0 || q.K < 0 || q.M > lim || q.N > lim || q.K > lim ||
            (reads && (!q.A || !q.B)) || q.lda < std::max<int64_t>(1, ta ? q.M : q.K) ||
            q.ldb < std::max<int64_t>(1, tb ? q.K : q.N) || (q.M > 0 && q.N > 0 && !q.C) ||
            q.ldc < std::max<int64_t>(1, q.N))
            return bad(100 + i);
    }

    auto* p = new gemm_grouped_plan_s();
    p->handle = h;
    p->device = gb300::handle_device(h);
    p->num_sms = gb300::handle_num_sms(h);
    p->err_word = gb300::handle_err_word(h);
    p->nterms = nterms;
    p->flags = flags;
    p->cfg = gb300::handle_tc_config(h, nterms);
    p->cfg.split_k = 1;
    // grouped CTA-pair kernels exist for the split-precision mode with bn 256
    if (p->cfg.cta_group == 2 && (nterms != 3 || p->cfg.bn != 256)) p->cfg.cta_group = 1;

    // Split placement.  The in-kernel split reads every A and B as stored
    // through FP32 tensor maps, so each must be 16-byte aligned with a row
    // stride that is a multiple of 4; it is considered when the handle asks
    // for it, or under GEMM_SPLIT_AUTO when the handle forces no tile shape.
    const int place = gb300::handle_split_place(h);
    bool aligned = true;
    for (int i = 0; i < count; ++i) {
        const gemm_problem_t& q = hp[i];
        if (q.M == 0 || q.N == 0 || q.K == 0 || q.alpha == 0.0f) continue;
        aligned = aligned && (reinterpret_cast<uintptr_t>(q.A) & 15) == 0 && q.lda % 4 == 0 &&
                  (reinterpret_cast<uintptr_t>(q.B) & 15) == 0 && q.ldb % 4 == 0;
    }
    const bool fused_ok = nterms == 3 && aligned && place != GEMM_SPLIT_PREPASS &&
                          (place == GEMM_SPLIT_IN_KERNEL || gb300::handle_tile_auto(h));
    const bool prepass_ok = !(fused_ok && place == GEMM_SPLIT_IN_KERNEL);
    if (fused_ok && !prepass_ok) {  // the in-kernel split's one tile shape
        p->cfg.fuse = 3;
        p->cfg.cta_group = 1;
        p->cfg.bn = 256;
        p->cfg.bk = 32;
        p->cfg.kmajor = 0;
    }

    // Workspace layout (split pass): per problem, the hi (and lo) planes of
    // A, then of B.  An operand stored K x rows (A with transA, B without
    // transB) keeps that orientation (MN-major tiles, split without
    // transposing) unless the handle asks for K-major operands.
    auto a_mn = [&](const gemm_problem_t& q) { return q.transA != 0 && !p->cfg.kmajor; };
    auto b_mn = [&](const gemm_problem_t& q) { return q.transB == 0 && !p->cfg.kmajor; };
    std::vector<HostProb> ps;    // operands as split-pass planes
    std::vector<HostProb> ps_f;  // the same problems with FP32 operands (in-kernel split)
    std::vector<SplitJob> jobs;
    std::vector<int> tile_job, tile_job_t;
    int tiles_t = 0;
    std::vector<size_t> a_off, b_off;
    size_t ws = 0;
    for (int i = 0; i < count; ++i) {
        const gemm_problem_t& q = hp[i];
        if (q.M == 0 || q.N == 0) continue;
        if (q.K == 0 || q.alpha == 0.0f) {
            p->scales.push_back({q.M, q.N, q.ldc, q.beta, q.C});
            continue;
        }
        HostProb hq;
        hq.M = q.M;
        hq.N = q.N;
        hq.K = q.K;
        hq.ldc = q.ldc;
        hq.alpha = q.alpha;
        hq.beta = q.beta;
        hq.C = q.C;
        if (fused_ok) {
            hq.a = TcOperand{nullptr, q.M, q.K, q.lda, 0, 2};
            hq.a.mn_major = q.transA != 0;
            hq.a.f32 = q.A;
            hq.b = TcOperand{nullptr, q.N, q.K, q.ldb, 0, 2};
            hq.b.mn_major = q.transB == 0;
            hq.b.f32 = q.B;
            ps_f.push_back(hq);
        }
        if (!prepass_ok) continue;
        a_off.push_back(ws);
        ws += round256(size_t(planes) * gb300::packed_layout(q.M, q.K, a_mn(q)).plane * 2);
        b_off.push_back(ws);
        ws += round256(size_t(planes) * gb300::packed_layout(q.N, q.K, b_mn(q)).plane * 2);
    }
    if (ws > 0 && cudaMalloc(reinterpret_cast<void**>(&p->ws), ws) != cudaSuccess) {
        cudaGetLastError();
        free_plan(p);
        return GEMM_ERR_WORKSPACE;
    }
    int tiles = 0;
    size_t idx = 0;
    for (int i = 0; i < count && prepass_ok; ++i) {
        const gemm_problem_t& q = hp[i];
        if (q.M == 0 || q.N == 0 || q.K == 0 || q.alpha == 0.0f) continue;
        uint16_t* ah = reinterpret_cast<uint16_t*>(p->ws + a_off[idx]);
        uint16_t* bh = reinterpret_cast<uint16_t*>(p->ws + b_off[idx]);
        ++idx;
        // One split job per operand: op(X) as rows x K (K-major, transposing
        // when X is stored K x rows) or X as stored, K x rows (MN-major).
        auto add_job = [&](const float* src, int64_t ldx, uint16_t* hi, int64_t rows,
                           bool stored_k_rows, bool mn) {
            const gb300::PackedLayout lay = gb300::packed_layout(rows, q.K, mn);
            SplitJob j{};
            j.src = src;
            j.ldx = ldx;
            j.hi = hi;
            j.lo = planes > 1 ? hi + lay.plane : nullptr;
            j.ldo = lay.ld;
            j.rows = int(mn ? q.K : rows);
            j.cols = int(mn ? rows : q.K);
            j.trans = (stored_k_rows && !mn) ? 1 : 0;
            j.x_vec = ((reinterpret_cast<uintptr_t>(src) & 15) == 0) && (ldx % 4 == 0);
            j.tiles_r = (j.rows + 63) / 64;
            const int tiles_c = (j.cols + 63) / 64;
            int& cnt = j.trans ? tiles_t : tiles;
            std::vector<int>& map = j.trans ? tile_job_t : tile_job;
            j.tile_start = cnt;
            cnt += j.tiles_r * tiles_c;
            map.insert(map.end(), size_t(j.tiles_r) * tiles_c, int(jobs.size()));
            jobs.push_back(j);
            TcOperand op{hi, rows, q.K, lay.ld, lay.plane, planes};
            op.mn_major = mn ? 1 : 0;
            return op;
        };
        HostProb hq;
        hq.a = add_job(q.A, q.lda, ah, q.M, q.transA != 0, a_mn(q));
        hq.b = add_job(q.B, q.ldb, bh, q.N, q.transB == 0, b_mn(q));
        hq.M = q.M;
        hq.N = q.N;
        hq.K = q.K;
        hq.ldc = q.ldc;
        hq.alpha = q.alpha;
        hq.beta = q.beta;
        hq.C = q.C;
        ps.push_back(hq);
    }
    p->njobs = int(jobs.size());
    p->split_tiles = tiles;
    p->split_tiles_t = tiles_t;
    p->nprobs = int(prepass_ok ? ps.size() : ps_f.size());
    gemm_status_t st = upload(&p->d_jobs, jobs, s);
    if (st == GEMM_OK) st = upload(&p->d_tile_job, tile_job, s);
    if (st == GEMM_OK) st = upload(&p->d_tile_job_t, tile_job_t, s);
    if (st != GEMM_OK) {
        free_plan(p);
        return st;
    }
    const std::vector<HostProb>& shapes = prepass_ok ? ps : ps_f;

    if (!(flags & GEMM_GROUPED_AUTOTUNE) && !shapes.empty() && gb300::handle_tile_auto(h)) {
        // library choice without timing: the analytic model's best
        // configuration and split placement
        const std::vector<Candidate> cands =
            seed_candidates(shapes, nterms, p->num_sms, p->cfg, prepass_ok, fused_ok);
        if (!cands.empty()) p->cfg = cands.front().cfg;
    }
    // straggler split-K unless the handle sets split_k 1 (never) or the
    // autotuner decides (below)
    const bool may_split = gb300::handle_split_k(h) != 1;
    p->cfg.split_k = may_split ? 2 : 1;
    if ((flags & GEMM_GROUPED_AUTOTUNE) && !shapes.empty()) {
        const std::string key = shape_key(p->num_sms, nterms, shapes) +
                                (prepass_ok ? "-p" : "") + (fused_ok ? "-f" : "");
        TcLaunch hit = p->cfg;
        if (cache_lookup(key, &hit)) {
            p->cfg.bn = hit.bn;
            p->cfg.bk = hit.bk;
            p->cfg.stages = hit.stages;
            p->cfg.raster_group = hit.raster_group;
            p->cfg.cta_group = hit.cta_group;
            p->cfg.fuse = hit.fuse;
            p->cfg.split_k = may_split ? hit.split_k : 1;
            if (hit.fuse) p->cfg.kmajor = 0;
        } else {
            // Operands must be split before the pre-split candidates can be
            // timed; the pass's own time is added to theirs, so that both
            // placements are compared over a whole plan run.
            double split_ms = 0.0;
            if (prepass_ok) {
                cudaEvent_t e0 = nullptr, e1 = nullptr;
                const bool ev = cudaEventCreate(&e0) == cudaSuccess &&
                                cudaEventCreate(&e1) == cudaSuccess;
                for (int rep = 0; rep < 2; ++rep) {  // the second run is timed
                    if (ev) cudaEventRecord(e0, s);
                    if (gb300::launch_split_grouped(p->d_jobs, p->d_tile_job, p->njobs,
                                                    p->split_tiles, p->num_sms, s) != cudaSuccess ||
                        gb300::launch_split_grouped_t(p->d_jobs, p->d_tile_job_t, p->njobs,
                                                      p->split_tiles_t, p->num_sms,
                                                      s) != cudaSuccess) {
                        if (e0) cudaEventDestroy(e0);
                        if (e1) cudaEventDestroy(e1);
                        free_plan(p);
                        return GEMM_ERR_CUDA;
                    }
                    if (ev) cudaEventRecord(e1, s);
                }
                float ms = 0.0f;
                if (ev && cudaEventSynchronize(e1) == cudaSuccess &&
                    cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                    split_ms = ms;
                cudaGetLastError();
                if (e0) cudaEventDestroy(e0);
                if (e1) cudaEventDestroy(e1);
            }
            // Tune on the whole problem set when its outputs fit in scratch of at
            // most 4 GB and a quarter of the free device memory (the wave count
            // of the persistent grid, which the timing must see, depends on the
            // whole set); otherwise on the leading problems that fit.
            size_t free_b = 0, total_b = 0;
            if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
                cudaGetLastError();
                free_b = 0;
            }
            const size_t tune_cap =
                std::max<size_t>(size_t(512) << 20, std::min<size_t>(size_t(4) << 30, free_b / 4));
            std::vector<HostProb> sub, sub_f;
            size_t cbytes = 0;
            for (size_t i = 0; i < shapes.size(); ++i) {
                const HostProb& q = shapes[i];
                const size_t b = round256(size_t(q.M) * q.N * 4);
                if (!sub.empty() && cbytes + b > tune_cap) break;
                sub.push_back(prepass_ok ? ps[i] : ps_f[i]);
                if (fused_ok) sub_f.push_back(ps_f[i]);
                cbytes += b;
            }
            uint8_t* scratch = nullptr;
            if (cudaMalloc(reinterpret_cast<void**>(&scratch), cbytes) != cudaSuccess) {
                cudaGetLastError();
                free_plan(p);
                return GEMM_ERR_WORKSPACE;
            }
            size_t off = 0;
            for (size_t i = 0; i < sub.size(); ++i) {
                for (std::vector<HostProb>* v : {&sub, &sub_f}) {
                    if (i >= v->size()) continue;
                    HostProb& q = (*v)[i];
                    q.C = reinterpret_cast<float*>(scratch + off);
                    q.ldc = q.N;
                    q.alpha = 1.0f;
                    q.beta = 0.0f;
                }
                off += round256(size_t(sub[i].M) * sub[i].N * 4);
            }
            // the split pass covers the whole set; scale its time to the subset
            const double frac = split_pass_seconds(sub) / std::max(1e-30, split_pass_seconds(shapes));
            std::vector<Candidate> cands =
                seed_candidates(sub, nterms, p->num_sms, p->cfg, prepass_ok, fused_ok);
            double best = -1.0;
            TcLaunch best_cfg = p->cfg;
            // the model's four best, plus the best of the placement it ranks lower
            std::vector<Candidate> tries(cands.begin(),
                                         cands.begin() + std::min<size_t>(cands.size(), 4));
            for (const Candidate& c : cands)
                if (c.cfg.fuse != tries.front().cfg.fuse) {
                    bool have = false;
                    for (const Candidate& t : tries) have = have || t.cfg.fuse == c.cfg.fuse;
                    if (!have) tries.push_back(c);
                    break;
                }
            for (const Candidate& cand : tries) {
                for (int rg : {8, 16}) {
                    TcLaunch cfg = cand.cfg;
                    cfg.raster_group = rg;
                    const double ms = time_candidate(cfg.fuse ? sub_f : sub, nterms, cfg,
                                                     p->err_word, p->num_sms, s);
                    const double total = ms + (cfg.fuse ? 0.0 : split_ms * frac);
                    if (ms > 0.0 && (best < 0.0 || total < best)) {
                        best = total;
                        best_cfg = cfg;
                    }
                }
            }
            // the best configuration with its straggler problems split along K
            // (the pre-split placement only), kept if faster
            best_cfg.split_k = 1;
            if (best > 0.0 && !best_cfg.fuse && may_split) {
                const double ms =
                    time_split_variant(sub, nterms, best_cfg, p->err_word, p->num_sms, s);
                if (ms > 0.0 && ms + split_ms * frac < best) {
                    best = ms + split_ms * frac;
                    best_cfg.split_k = 2;
                }
            }
            cudaFree(scratch);
            if (best > 0.0) {
                p->cfg = best_cfg;
                p->tuned_ms = best;
                cache_store(key, best_cfg);
            }
        }
    }
    if (p->cfg.fuse) {
        // no split pass: drop its workspace and tables
        if (p->ws) cudaFree(p->ws);
        p->ws = nullptr;
        p->njobs = p->split_tiles = p->split_tiles_t = 0;
        p->nprobs = int(ps_f.size());
    }

    // per-problem split-K of the straggler problems (pre-split placement)
    std::vector<HostProb> sliced;
    const std::vector<HostProb>* run_ps = p->cfg.fuse ? &ps_f : &ps;
    if (!p->cfg.fuse && p->cfg.split_k > 1 && !ps.empty()) {
        const std::vector<int> splits = straggler_splits(ps, p->cfg, p->num_sms);
        const int most = *std::max_element(splits.begin(), splits.end());
        if (most > 1) {
            const size_t floats = slice_problems(ps, splits, p->cfg.bk, nullptr, &sliced, nullptr);
            if (cudaMalloc(reinterpret_cast<void**>(&p->partials), floats * sizeof(float)) !=
                cudaSuccess) {
                cudaGetLastError();
                free_plan(p);
                return GEMM_ERR_WORKSPACE;
            }
            slice_problems(ps, splits, p->cfg.bk, p->partials, &sliced, &p->reduces);
            std::vector<gb300::ReduceJob> rjobs;
            p->reduce_units = reduce_table(p->reduces, &rjobs);
            if ((st = upload(&p->d_reduces, rjobs, s)) != GEMM_OK) {
                free_plan(p);
                return st;
            }
            run_ps = &sliced;
            p->nprobs = int(sliced.size());
            p->max_split = most;
        }
    }
    p->cfg.split_k = 1;  // the grouped kernel itself never slices K
    std::vector<GroupedProblem> probs;
    std::vector<CUtensorMap> maps;
    std::vector<int> tile_prob;
    bool ok = true;
    p->total_tiles = build_tables(*run_ps, p->cfg, probs, maps, tile_prob, &ok);
    if (!ok) {
        free_plan(p);
        return GEMM_ERR_CUDA;
    }
    if ((st = upload(&p->d_probs, probs, s)) != GEMM_OK ||
        (st = upload(&p->d_maps, maps, s)) != GEMM_OK ||
        (st = upload(&p->d_tile_prob, tile_prob, s)) != GEMM_OK) {
        free_plan(p);
        return st;
    }
    p->launches = int(p->scales.size()) + (p->split_tiles > 0 ? 1 : 0) +
                  (p->split_tiles_t > 0 ? 1 : 0) + (p->nprobs > 0 ? 1 : 0) +
                  (p->reduces.empty() ? 0 : 1);
    *plan = p;
    return GEMM_OK;
}

gemm_status_t gemm_grouped_plan_run(gemm_grouped_plan_t p, void* stream) {
    if (!p) return GEMM_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    gb300::handle_set_launches(p->handle, p->launches);
    if (!(p->flags & GEMM_GROUPED_GRAPH) || s == nullptr) return enqueue(p, s);
    if (!p->exec) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return GEMM_ERR_CUDA;
        const gemm_status_t st = enqueue(p, s);
        const cudaError_t ce = cudaStreamEndCapture(s, &graph);
        if (st != GEMM_OK || ce != cudaSuccess || !graph) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return st != GEMM_OK ? st : GEMM_ERR_CUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&p->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            p->exec = nullptr;
            cudaGetLastError();
            return GEMM_ERR_CUDA;
        }
    }
    return cudaGraphLaunch(p->exec, s) == cudaSuccess ? GEMM_OK : GEMM_ERR_CUDA;
}

gemm_status_t gemm_grouped_plan_config(gemm_grouped_plan_t p, gemm_config_t* cfg,
                                       double* tuned_ms) {
    if (!p) return GEMM_ERR_ARG;
    if (cfg) {
        *cfg = gemm_config_t{};
        cfg->bn = p->cfg.bn;
        cfg->bk = p->cfg.bk;
        cfg->stages = p->cfg.stages;
        cfg->split_k = p->max_split;  // the most slices of any problem (1: none split)
        cfg->raster_group = p->cfg.raster_group;
        cfg->max_ctas = p->cfg.max_ctas;
        cfg->promote_k = p->cfg.promote_k > 0 ? p->cfg.promote_k : -1;
        cfg->cta_group = p->cfg.cta_group;
        cfg->wait_poll_limit = p->cfg.poll_limit;
        cfg->operand_layout = p->cfg.kmajor ? GEMM_LAYOUT_K_MAJOR : GEMM_LAYOUT_AS_STORED;
        cfg->split_place = p->cfg.fuse ? GEMM_SPLIT_IN_KERNEL : GEMM_SPLIT_PREPASS;
    }
    if (tuned_ms) *tuned_ms = p->tuned_ms;
    return GEMM_OK;
}

gemm_status_t gemm_grouped_plan_destroy(gemm_grouped_plan_t p) {
    if (!p) return GEMM_OK;
    cudaDeviceSynchronize();
    free_plan(p);
    return GEMM_OK;
}

gemm_status_t gemm_grouped(gemm_handle_t h, gemm_mode_t mode, const gemm_problem_t* host_problems,
                           int32_t count, void* stream) {
    gemm_grouped_plan_t plan = nullptr;
    gemm_status_t st = gemm_grouped_plan_create(h, mode, host_problems, count, 0, stream, &plan);
    if (st != GEMM_OK) return st;
    st = gemm_grouped_plan_run(plan, stream);
    gemm_grouped_plan_destroy(plan);
    return st;
}

}  // extern "C"
