// C-ABI entry points (include/rankfhe.h): argument checks, exception-to-status
// translation and handle ownership.  All compute is in the CUDA kernels.
#include <cstring>

#include "kernels.cuh"

void ctx_build(rk_ctx* c, const rk_params* p, int device, void* stream);
void ctx_release(rk_ctx* c);
rk_ct* circuit_rank(rk_ctx* c, const rk_ct* in, uint32_t flags);
rk_ct* circuit_compare_matrix(rk_ctx* c, const rk_ct* in);
void rescale_noalloc(rk_ctx* c, const u64* in, u64* out, int l);
rk_ct* circuit_order_stat(rk_ctx* c, const rk_ct* in, uint32_t k, uint32_t flags);
rk_ct* circuit_order_value_all(rk_ctx* c, const rk_ct* in, uint32_t k);
rk_ct* circuit_sort(rk_ctx* c, const rk_ct* in, uint32_t flags);
rk_ct* circuit_order_value(rk_ctx* c, const rk_ct* in, uint32_t k);
rk_ct* circuit_median(rk_ctx* c, const rk_ct* in);
void indicator_import(rk_ctx* c, uint32_t N, const double* coeffs, size_t count);
void circuit_rank_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs);
void circuit_rank_blocked_partial(rk_ctx* c, const rk_ct* const* blocks, int L, const std::vector<std::pair<int, int>>& pairs,
                                  rk_ct** A_out, rk_ct** B_out);
void circuit_rank_blocked_finish(rk_ctx* c, const rk_ct* const* A_in, const rk_ct* const* B_in, int L, rk_ct** outs);
void circuit_rank_blocked_tc(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs);
void circuit_order_stat_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, uint32_t k, rk_ct** outs);
void circuit_sort_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs);
rk_graph* graph_rank_capture(rk_ctx* c, const rk_ct* tmpl, uint32_t flags);
rk_graph* graph_capture(rk_ctx* c, uint32_t op, uint32_t arg, uint32_t flags, int L, const rk_ct* tmpl);
rk_server* server_start(rk_ctx* c, size_t budget, int max_stack);
uint64_t server_submit(rk_ctx* c, uint32_t op, uint32_t arg, uint32_t flags, const rk_ct* in);
rk_ct* server_collect(rk_ctx* c, uint64_t ticket, double timeout_s);
void server_stats(rk_ctx* c, double out[8]);
void ntt_autotune(rk_ctx* c, std::vector<double>& report);
void ks_autotune(rk_ctx* c, std::vector<double>& report);
size_t server_latencies(rk_ctx* c, double* out, size_t cap);
void server_stop(rk_ctx* c);
void server_stats_lanes(rk_ctx* c, double out[5]);
rk_ct* graph_rank_run(rk_graph* g, const rk_ct* in);
void graph_free(rk_graph* g);
rk_ctx* graph_context(const rk_graph* g);
void circuit_rotations(uint32_t N, std::vector<int>& out);
void measure_alu(rk_ctx* c, double out[5]);
void params_chain(const rk_params* p, std::vector<u64>& primes, std::vector<double>& scales);

namespace {
thread_local std::string g_last_error;

template <class F>
rk_status guard(F&& f) {
    try {
        f();
        return RK_OK;
    } catch (const rk_error& e) {
        g_last_error = e.what();
        return e.code;
    } catch (const std::bad_alloc&) {
        g_last_error = "host allocation failed";
        return RK_ENOMEM;
    } catch (const std::exception& e) {
        g_last_error = e.what();
        return RK_EINVAL;
    }
}

void need(const void* p, const char* what) {
    if (!p) throw rk_error(RK_EINVAL, std::string(what) + " is NULL");
}

void same_ctx(const rk_ctx* c, const rk_ct* a) {
    need(a, "ciphertext");
    if (a->ctx != c) throw rk_error(RK_EINVAL, "ciphertext belongs to another context");
}

void set_device(rk_ctx* c) { RK_CUDA(cudaSetDevice(c->device)); }

// Check for a launch error after queuing kernels.
void check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw rk_error(RK_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
}
}  // namespace

// Queries of one level and vector shape are stacked and run as one circuit.
template <class F>
static void run_grouped(rk_ctx* ctx, const rk_ct* const* in, size_t count, rk_ct** out, F circuit) {
    std::map<std::tuple<int, uint32_t, uint32_t, uint32_t, uint32_t>, std::vector<size_t>> groups;
    for (size_t i = 0; i < count; i++) {
        same_ctx(ctx, in[i]);
        RK_REQUIRE(in[i]->B == 1, RK_EINVAL, "batched calls take single ciphertexts");
        groups[std::make_tuple(in[i]->level, in[i]->N, in[i]->Q, in[i]->n_real, in[i]->layout)].push_back(i);
    }
    std::vector<rk_ct*> res(count, nullptr);
    try {
        for (auto& g : groups) {
            std::vector<const rk_ct*> members;
            for (size_t i : g.second) members.push_back(in[i]);
            rk_ct* st = ct_stack(ctx, members.data(), (int)members.size());
            rk_ct* r = nullptr;
            try {
                r = circuit(st);
            } catch (...) {
                ct_free(st);
                throw;
            }
            ct_free(st);
            std::vector<rk_ct*> parts(members.size());
            ct_unstack(ctx, r, parts.data());
            ct_free(r);
            for (size_t k = 0; k < g.second.size(); k++) res[g.second[k]] = parts[k];
        }
        check_launch();
    } catch (...) {
        for (auto* p : res) ct_free(p);
        throw;
    }
    for (size_t i = 0; i < count; i++) out[i] = res[i];
}

extern "C" {

const char* rk_last_error(void) { return g_last_error.c_str(); }

rk_status rk_ctx_create(const rk_params* params, int device, void* cuda_stream, rk_ctx** out) {
    return guard([&] {
        need(out, "out");
        *out = nullptr;
        rk_ctx* c = new rk_ctx();
        try {
            ctx_build(c, params, device, cuda_stream);
        } catch (...) {
            ctx_release(c);
            delete c;
            throw;
        }
        *out = c;
    });
}

void rk_ctx_destroy(rk_ctx* ctx) {
    if (!ctx) return;
    ctx_release(ctx);
    delete ctx;
}

rk_status rk_ctx_moduli(const rk_ctx* ctx, uint64_t* out, size_t cap, size_t* count) {
    return guard([&] {
        need(ctx, "ctx");
        if (count) *count = ctx->primes.size();
        if (out)
            for (size_t i = 0; i < ctx->primes.size() && i < cap; i++) out[i] = ctx->primes[i];
    });
}

rk_status rk_params_chain(const rk_params* params, uint64_t* moduli, size_t cap, size_t* count, double* scales,
                          size_t scales_cap) {
    return guard([&] {
        need(params, "params");
        std::vector<u64> q;
        std::vector<double> sc;
        params_chain(params, q, sc);
        if (count) *count = q.size();
        if (moduli)
            for (size_t i = 0; i < q.size() && i < cap; i++) moduli[i] = q[i];
        if (scales)
            for (size_t i = 0; i < sc.size() && i < scales_cap; i++) scales[i] = sc[i];
    });
}

rk_status rk_ctx_scales(const rk_ctx* ctx, double* out, size_t cap) {
    return guard([&] {
        need(ctx, "ctx");
        need(out, "out");
        for (size_t i = 0; i < ctx->scales.size() && i < cap; i++) out[i] = ctx->scales[i];
    });
}

rk_status rk_sync(rk_ctx* ctx) {
    return guard([&] {
        need(ctx, "ctx");
        RK_CUDA(cudaStreamSynchronize(ctx->stream));
    });
}

rk_status rk_ctx_counters(const rk_ctx* ctx, uint64_t out[4]) {
    return guard([&] {
        need(ctx, "ctx");
        need(out, "out");
        out[0] = ctx->n_ks;
        out[1] = ctx->n_rot;
        out[2] = ctx->n_mul;
        out[3] = ctx->n_rescale;
    });
}

rk_status rk_ctx_set_option(rk_ctx* ctx, uint32_t option, int64_t value) {
    return guard([&] {
        need(ctx, "ctx");
        RK_REQUIRE(value >= 0, RK_EINVAL, "option value must be non-negative");
        RK_CUDA(cudaStreamSynchronize(ctx->stream));
        switch (option) {
            case RK_OPT_KS_FUSED: ctx->ks_fused = value != 0; break;
            case RK_OPT_KS_GROUP_BYTES: ctx->ks_group_bytes = (double)value; break;
            case RK_OPT_BLOCK_STACKING: ctx->stack_blocks = value != 0; break;
            case RK_OPT_TRIM_LEVELS: ctx->trim_levels = value != 0; break;
            case RK_OPT_PAIR_PACKING: ctx->pair_packing = value != 0; break;
            case RK_OPT_STACK_BUDGET:
                RK_REQUIRE(value >= 1, RK_EINVAL, "stack budget must be positive");
                ctx->stack_budget_bytes = (size_t)value;
                break;
            case RK_OPT_INDICATOR_BUDGET:
                RK_REQUIRE(value >= 1, RK_EINVAL, "indicator budget must be positive");
                ctx->ind_stack_bytes = (size_t)value;
                break;
            case RK_OPT_MODUP_COL: ctx->modup_col = value != 0; break;
            case RK_OPT_NTT_GROUP_BYTES:
                RK_REQUIRE(value >= 0, RK_EINVAL, "NTT group bytes must not be negative");
                ctx->tune.ntt_group_bytes = (size_t)value;
                break;
            case RK_OPT_SERVER_LANES:
                RK_REQUIRE(value >= 1 && value <= 16, RK_EINVAL, "server lanes must be 1 to 16");
                ctx->server_lanes = (int)value;
                break;
            default: throw rk_error(RK_EINVAL, "unknown option " + std::to_string(option));
        }
    });
}

rk_status rk_autotune(rk_ctx* ctx, double* report, size_t cap, size_t* count) {
    return guard([&] {
        need(ctx, "ctx");
        RK_REQUIRE(!ctx->server, RK_EINVAL, "autotune while a server runs");
        set_device(ctx);
        std::vector<double> rep;
        ntt_autotune(ctx, rep);
        ks_autotune(ctx, rep);
        if (report)
            for (size_t i = 0; i < std::min(cap, rep.size()); i++) report[i] = rep[i];
        if (count) *count = rep.size();
    });
}

rk_status rk_keygen(rk_ctx* ctx, uint64_t seed, uint32_t max_len) {
    return guard([&] {
        need(ctx, "ctx");
        set_device(ctx);
        RK_REQUIRE((size_t)max_len * max_len <= (size_t)ctx->n / 2, RK_EINVAL, "max_len^2 exceeds the slots");
        std::vector<int> rots;
        for (uint32_t N = 2; N <= max_len; N <<= 1) circuit_rotations(N, rots);
        keys_generate(ctx, seed, rots);
        check_launch();
    });
}

rk_status rk_keygen_rotations(rk_ctx* ctx, const int32_t* r, size_t count) {
    return guard([&] {
        need(ctx, "ctx");
        need(r, "r");
        set_device(ctx);
        keys_add_rotations(ctx, std::vector<int>(r, r + count));
        check_launch();
    });
}

rk_status rk_secret_import(rk_ctx* ctx, const int64_t* s, size_t n) {
    return guard([&] {
        need(ctx, "ctx");
        need(s, "s");
        set_device(ctx);
        secret_import(ctx, s, n);
        check_launch();
    });
}

rk_status rk_key_import(rk_ctx* ctx, uint32_t kind, uint64_t galois, const uint64_t* coeffs, size_t words) {
    return guard([&] {
        need(ctx, "ctx");
        need(coeffs, "coeffs");
        set_device(ctx);
        key_import(ctx, kind, galois, coeffs, words);
        check_launch();
    });
}

rk_status rk_key_import_seeded(rk_ctx* ctx, uint32_t kind, uint64_t galois, uint64_t seed, const uint64_t* coeffs, size_t words) {
    return guard([&] {
        need(ctx, "ctx");
        need(coeffs, "coeffs");
        set_device(ctx);
        key_import(ctx, kind, galois, coeffs, words, true, seed);
        check_launch();
    });
}

uint64_t rk_galois_left(const rk_ctx* ctx, int32_t r) { return ctx ? galois_left(ctx, r) : 0; }

rk_status rk_encoding_import(rk_ctx* ctx, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real, const double* u, size_t n) {
    return guard([&] {
        need(ctx, "ctx");
        need(u, "u");
        RK_REQUIRE(n == (size_t)ctx->n, RK_EINVAL, "encoding length must be n");
        RK_REQUIRE(kind >= RK_MASK_ROW0 && kind <= RK_MASK_ROWIDX, RK_EINVAL, "unknown mask kind");
        const uint32_t nr = mask_nreal(kind, n_real);
        ctx->encodings[std::make_tuple(kind, N, Q, nr)] = std::vector<double>(u, u + n);
        ctx->generation++;
        for (auto* cache : {&ctx->plain_cache, &ctx->plain_add_cache})
            for (auto it = cache->begin(); it != cache->end();) {
                if (std::get<0>(it->first) == kind && std::get<1>(it->first) == N && std::get<2>(it->first) == Q &&
                    std::get<3>(it->first) == nr) {
                    cudaFree(it->second);
                    it = cache->erase(it);
                } else {
                    ++it;
                }
            }
    });
}

uint64_t rk_device_alloc_count(void) { return rk_alloc_counted(); }

rk_status rk_measure_alu(rk_ctx* ctx, double out[5]) {
    return guard([&] {
        need(ctx, "ctx");
        need(out, "out");
        set_device(ctx);
        measure_alu(ctx, out);
    });
}

rk_status rk_encoding_export(rk_ctx* ctx, uint32_t kind, uint32_t N, uint32_t Q, uint32_t n_real, double* u, size_t n) {
    return guard([&] {
        need(ctx, "ctx");
        need(u, "u");
        RK_REQUIRE(n == (size_t)ctx->n, RK_EINVAL, "encoding length must be n");
        RK_REQUIRE(kind >= RK_MASK_ROW0 && kind <= RK_MASK_ROWIDX, RK_EINVAL, "unknown mask kind");
        RK_REQUIRE(N >= 1 && (N & (N - 1)) == 0 && Q >= 1 && (size_t)Q * N * N <= (size_t)ctx->n / 2, RK_EINVAL,
                   "N must be a power of two with Q N^2 <= n/2");
        const std::vector<double>& e = encoding_of(ctx, kind, N, Q, mask_nreal(kind, n_real));
        std::copy(e.begin(), e.end(), u);
    });
}

static void copy_coeffs(const std::vector<double>& c, double* out, size_t cap, size_t* count) {
    *count = c.size();
    if (out) std::copy(c.begin(), c.begin() + std::min(cap, c.size()), out);
}

rk_status rk_indicator_export(rk_ctx* ctx, uint32_t N, double* out, size_t cap, size_t* count) {
    return guard([&] {
        need(ctx, "ctx");
        need(count, "count");
        RK_REQUIRE(N >= 1 && (N & (N - 1)) == 0, RK_EINVAL, "N must be a power of two");
        copy_coeffs(indicator_coeffs_of(ctx, N), out, cap, count);
    });
}

rk_status rk_comparator_export(rk_ctx* ctx, double* out, size_t cap, size_t* count) {
    return guard([&] {
        need(ctx, "ctx");
        need(count, "count");
        copy_coeffs(comparator_coeffs_of(ctx), out, cap, count);
    });
}

rk_status rk_encrypt(rk_ctx* ctx, const double* v, uint32_t count, uint32_t N, uint32_t Q, uint32_t n_real, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        need(out, "out");
        need(v, "v");
        set_device(ctx);
        *out = encrypt_values(ctx, v, count, N, Q, n_real);
        check_launch();
    });
}

rk_status rk_decrypt_slots(rk_ctx* ctx, const rk_ct* ct, double* out, size_t cap) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, ct);
        need(out, "out");
        set_device(ctx);
        std::vector<double> s;
        decrypt_slots(ctx, ct, s);
        for (size_t i = 0; i < s.size() && i < cap; i++) out[i] = s[i];
    });
}

rk_status rk_decrypt(rk_ctx* ctx, const rk_ct* ct, double* out, size_t cap, uint32_t* n_out) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, ct);
        set_device(ctx);
        std::vector<double> s;
        decrypt_slots(ctx, ct, s);
        const size_t NN = (size_t)ct->N * ct->N;
        size_t w = 0;
        for (uint32_t q = 0; q < ct->Q; q++)
            for (uint32_t i = 0; i < ct->n_real; i++) {
                size_t slot = q * NN + (ct->layout == RK_LAYOUT_COL ? (size_t)i * ct->N : i);
                if (out && w < cap) out[w] = s[slot];
                w++;
            }
        if (n_out) *n_out = (uint32_t)w;
    });
}

rk_status rk_ct_import(rk_ctx* ctx, const uint64_t* coeffs, uint32_t level, uint32_t N, uint32_t Q, uint32_t n_real,
                       rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        need(coeffs, "coeffs");
        need(out, "out");
        RK_REQUIRE(N >= 1 && (N & (N - 1)) == 0 && n_real >= 1 && n_real <= N && Q >= 1, RK_EINVAL, "bad vector metadata");
        set_device(ctx);
        rk_ct* ct = ct_import(ctx, coeffs, (int)level);
        ct->N = N;
        ct->Q = Q;
        ct->n_real = n_real;
        ct->layout = RK_LAYOUT_ROW;
        *out = ct;
    });
}

rk_status rk_ct_export(const rk_ct* ct, uint64_t* coeffs, size_t cap) {
    return guard([&] {
        need(ct, "ct");
        need(coeffs, "coeffs");
        rk_ctx* c = ct->ctx;
        RK_REQUIRE(cap >= (size_t)2 * (ct->level + 1) * c->n, RK_EINVAL, "export buffer too small");
        set_device(c);
        ct_export(c, ct, coeffs);
    });
}

uint32_t rk_ct_level(const rk_ct* ct) { return ct ? (uint32_t)ct->level : 0; }

void rk_ct_free(rk_ct* ct) {
    if (ct) ct_free(ct);
}

#define RK_UNARY_OUT(ctx, a, out, level_expr, body) \
    need(ctx, "ctx");                                 \
    same_ctx(ctx, a);                                 \
    need(out, "out");                                 \
    set_device(ctx);                                  \
    rk_ct* o = ct_clone_meta(a, (level_expr));        \
    try {                                             \
        body;                                         \
        check_launch();                               \
    } catch (...) {                                   \
        ct_free(o);                                   \
        throw;                                        \
    }                                                 \
    *out = o;

rk_status rk_rotate(rk_ctx* ctx, const rk_ct* in, int32_t r, rk_ct** out) {
    return guard([&] {
        RK_UNARY_OUT(ctx, in, out, in->level, {
            int rr = r;
            rk_ct* outs[1] = {o};
            ev_rotate_many(ctx, in, &rr, 1, outs);
        })
    });
}

rk_status rk_rotate_many(rk_ctx* ctx, const rk_ct* in, const int32_t* r, uint32_t k, rk_ct** outs) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, in);
        need(r, "r");
        need(outs, "outs");
        set_device(ctx);
        std::vector<rk_ct*> o(k);
        std::vector<int> rr(r, r + k);
        for (uint32_t i = 0; i < k; i++) o[i] = ct_clone_meta(in, in->level);
        try {
            ev_rotate_many(ctx, in, rr.data(), (int)k, o.data());
            check_launch();
        } catch (...) {
            for (auto* p : o) ct_free(p);
            throw;
        }
        for (uint32_t i = 0; i < k; i++) outs[i] = o[i];
    });
}

rk_status rk_add(rk_ctx* ctx, const rk_ct* a, const rk_ct* b, rk_ct** out) {
    return guard([&] {
        same_ctx(ctx, b);
        RK_UNARY_OUT(ctx, a, out, a->level, ev_add(ctx, a, b, o))
    });
}

rk_status rk_sub(rk_ctx* ctx, const rk_ct* a, const rk_ct* b, rk_ct** out) {
    return guard([&] {
        same_ctx(ctx, b);
        RK_UNARY_OUT(ctx, a, out, a->level, ev_sub(ctx, a, b, o))
    });
}

rk_status rk_add_const(rk_ctx* ctx, const rk_ct* a, double v, rk_ct** out) {
    return guard([&] { RK_UNARY_OUT(ctx, a, out, a->level, ev_add_const(ctx, a, v, o)) });
}

rk_status rk_mul(rk_ctx* ctx, const rk_ct* a, const rk_ct* b, rk_ct** out) {
    return guard([&] {
        same_ctx(ctx, b);
        RK_UNARY_OUT(ctx, a, out, a->level, ev_mul(ctx, a, b, o))
    });
}

rk_status rk_mul_scalar(rk_ctx* ctx, const rk_ct* a, double v, rk_ct** out) {
    return guard([&] { RK_UNARY_OUT(ctx, a, out, a->level, ev_mul_scalar(ctx, a, v, o)) });
}

rk_status rk_mul_mask(rk_ctx* ctx, const rk_ct* a, uint32_t kind, rk_ct** out) {
    return guard([&] {
        RK_REQUIRE(kind >= RK_MASK_ROW0 && kind <= RK_MASK_ROWIDX, RK_EINVAL, "unknown mask kind");
        RK_UNARY_OUT(ctx, a, out, a->level,
                     ev_mul_plain(ctx, a, kind, a->N, a->Q, kind == RK_MASK_VALID ? a->n_real : 0, o))
    });
}

rk_status rk_rescale(rk_ctx* ctx, const rk_ct* a, rk_ct** out) {
    return guard([&] {
        RK_UNARY_OUT(ctx, a, out, a->level, {
            ev_copy(ctx, a, o);
            ev_rescale_inplace(ctx, o);
        })
    });
}

rk_status rk_rank(rk_ctx* ctx, const rk_ct* in, uint32_t flags, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, in);
        need(out, "out");
        set_device(ctx);
        *out = circuit_rank(ctx, in, flags);
        check_launch();
    });
}

rk_status rk_indicator_import(rk_ctx* ctx, uint32_t N, const double* coeffs, size_t count) {
    return guard([&] {
        need(ctx, "ctx");
        need(coeffs, "coeffs");
        indicator_import(ctx, N, coeffs, count);
    });
}

rk_status rk_order_value_all(rk_ctx* ctx, const rk_ct* in, uint32_t k, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, in);
        need(out, "out");
        RK_REQUIRE(k >= 1 && k <= in->N, RK_EINVAL, "k must be in [1, N]");
        set_device(ctx);
        *out = circuit_order_value_all(ctx, in, k);
        check_launch();
    });
}

rk_status rk_order_stat(rk_ctx* ctx, const rk_ct* in, uint32_t k, uint32_t flags, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, in);
        need(out, "out");
        set_device(ctx);
        *out = circuit_order_stat(ctx, in, k, flags);
        check_launch();
    });
}

rk_status rk_sort(rk_ctx* ctx, const rk_ct* in, uint32_t flags, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, in);
        need(out, "out");
        set_device(ctx);
        *out = circuit_sort(ctx, in, flags);
        check_launch();
    });
}

rk_status rk_order_value(rk_ctx* ctx, const rk_ct* in, uint32_t k, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, in);
        need(out, "out");
        set_device(ctx);
        RK_REQUIRE(k >= 1 && k <= in->N, RK_EINVAL, "k must be in [1, N]");
        *out = circuit_order_value(ctx, in, k);
        check_launch();
    });
}

rk_status rk_median(rk_ctx* ctx, const rk_ct* in, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, in);
        need(out, "out");
        set_device(ctx);
        *out = circuit_median(ctx, in);
        check_launch();
    });
}

rk_status rk_compare_matrix(rk_ctx* ctx, const rk_ct* in, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, in);
        need(out, "out");
        set_device(ctx);
        *out = circuit_compare_matrix(ctx, in);
        check_launch();
    });
}

rk_status rk_rank_batch(rk_ctx* ctx, const rk_ct* const* in, size_t count, uint32_t flags, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        need(in, "in");
        need(out, "out");
        set_device(ctx);
        run_grouped(ctx, in, count, out, [&](const rk_ct* st) { return circuit_rank(ctx, st, flags); });
    });
}

rk_status rk_order_stat_batch(rk_ctx* ctx, const rk_ct* const* in, size_t count, uint32_t k, uint32_t flags, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        need(in, "in");
        need(out, "out");
        set_device(ctx);
        run_grouped(ctx, in, count, out, [&](const rk_ct* st) { return circuit_order_stat(ctx, st, k, flags); });
    });
}

rk_status rk_sort_batch(rk_ctx* ctx, const rk_ct* const* in, size_t count, uint32_t flags, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        need(in, "in");
        need(out, "out");
        set_device(ctx);
        run_grouped(ctx, in, count, out, [&](const rk_ct* st) { return circuit_sort(ctx, st, flags); });
    });
}

// ---- key set blob: little-endian u64 words ----
//   magic, log_n, n_primes (L+1+alpha), beta_L, K, then K records
//   [kind][galois][seeded][seed][words][words x u64 in rk_key_import's layout, or
//   rk_key_import_seeded's when seeded]
static const uint64_t kKeysMagic = 0x32305359454b4b52ull;   // "RKKEYS02"

rk_status rk_comparator_import(rk_ctx* ctx, const double* coeffs, size_t count) {
    return guard([&] {
        need(ctx, "ctx");
        need(coeffs, "coeffs");
        RK_REQUIRE(ctx->prm.cmp_cheb != 0 && count == ctx->prm.cmp_cheb, RK_EINVAL,
                   "the context's comparator does not take this many Chebyshev coefficients");
        ctx->cmp_coeffs.assign(coeffs, coeffs + count);
        ctx->generation++;
    });
}

rk_status rk_keys_export(rk_ctx* ctx, uint8_t* buf, size_t cap, size_t* len) {
    return guard([&] {
        need(ctx, "ctx");
        need(len, "len");
        set_device(ctx);
        std::vector<std::pair<std::pair<uint64_t, uint64_t>, const SwitchKeyDev*>> keys;
        if (ctx->rlk.data) keys.push_back({{RK_KEY_RELIN, 0}, &ctx->rlk});
        for (auto& kv : ctx->gal) keys.push_back({{RK_KEY_GALOIS, kv.first}, &kv.second});
        size_t total = 8 * 5;
        for (auto& k : keys) total += 8 * (5 + key_words(ctx, *k.second));
        *len = total;
        if (!buf) return;
        RK_REQUIRE(cap >= total, RK_EINVAL, "buffer too small for the key set");
        uint64_t* w = reinterpret_cast<uint64_t*>(buf);
        RK_REQUIRE(reinterpret_cast<uintptr_t>(buf) % 8 == 0, RK_EINVAL, "buffer must be 8-byte aligned");
        w[0] = kKeysMagic;
        w[1] = (uint64_t)ctx->log_n;
        w[2] = (uint64_t)ctx->n_primes;
        w[3] = (uint64_t)ctx->beta(ctx->L);
        w[4] = keys.size();
        size_t at = 5;
        for (auto& k : keys) {
            const size_t words = key_words(ctx, *k.second);
            w[at] = k.first.first;
            w[at + 1] = k.first.second;
            w[at + 2] = k.second->seeded ? 1 : 0;
            w[at + 3] = k.second->seed;
            w[at + 4] = words;
            key_export(ctx, *k.second, reinterpret_cast<u64*>(w + at + 5));
            at += 5 + words;
        }
    });
}

rk_status rk_keys_import(rk_ctx* ctx, const uint8_t* buf, size_t len) {
    return guard([&] {
        need(ctx, "ctx");
        need(buf, "buf");
        set_device(ctx);
        RK_REQUIRE(len >= 40 && len % 8 == 0 && reinterpret_cast<uintptr_t>(buf) % 8 == 0, RK_EFORMAT,
                   "key set blob: bad length or alignment");
        const uint64_t* w = reinterpret_cast<const uint64_t*>(buf);
        const size_t nw = len / 8;
        RK_REQUIRE(w[0] == kKeysMagic, RK_EFORMAT, "key set blob: bad magic");
        RK_REQUIRE(w[1] == (uint64_t)ctx->log_n && w[2] == (uint64_t)ctx->n_primes && w[3] == (uint64_t)ctx->beta(ctx->L),
                   RK_EFORMAT, "key set blob: parameters differ from the context's");
        size_t at = 5;
        for (uint64_t k = 0; k < w[4]; k++) {
            RK_REQUIRE(at + 5 <= nw && at + 5 + w[at + 4] <= nw, RK_EFORMAT, "key set blob: truncated");
            RK_REQUIRE(w[at + 2] <= 1, RK_EFORMAT, "key set blob: bad seeded flag");
            key_import(ctx, (uint32_t)w[at], w[at + 1], w + at + 5, (size_t)w[at + 4], w[at + 2] == 1, w[at + 3]);
            at += 5 + (size_t)w[at + 4];
        }
    });
}

rk_status rk_rank_blocked(rk_ctx* ctx, const rk_ct* const* blocks, uint32_t L, uint32_t flags, rk_ct** outs) {
    return guard([&] {
        need(ctx, "ctx");
        need(blocks, "blocks");
        need(outs, "outs");
        RK_REQUIRE(flags == 0 || flags == RK_TIES_CORRECT, RK_EINVAL, "blocked rank flags: 0 or RK_TIES_CORRECT");
        for (uint32_t i = 0; i < L; i++) same_ctx(ctx, blocks[i]);
        set_device(ctx);
        if (flags & RK_TIES_CORRECT)
            circuit_rank_blocked_tc(ctx, blocks, (int)L, outs);
        else
            circuit_rank_blocked(ctx, blocks, (int)L, outs);
        check_launch();
    });
}

rk_status rk_rank_blocked_partial(rk_ctx* ctx, const rk_ct* const* blocks, uint32_t L, const uint32_t* pair_i,
                                  const uint32_t* pair_j, uint32_t npairs, rk_ct** A, rk_ct** B) {
    return guard([&] {
        need(ctx, "ctx");
        need(blocks, "blocks");
        need(A, "A");
        need(B, "B");
        RK_REQUIRE(npairs == 0 || (pair_i && pair_j), RK_EINVAL, "pair lists are NULL");
        for (uint32_t i = 0; i < L; i++) same_ctx(ctx, blocks[i]);
        std::vector<std::pair<int, int>> pairs;
        for (uint32_t p = 0; p < npairs; p++) pairs.push_back({(int)pair_i[p], (int)pair_j[p]});
        set_device(ctx);
        circuit_rank_blocked_partial(ctx, blocks, (int)L, pairs, A, B);
        check_launch();
    });
}

rk_status rk_rank_blocked_finish(rk_ctx* ctx, const rk_ct* const* A, const rk_ct* const* B, uint32_t L, rk_ct** outs) {
    return guard([&] {
        need(ctx, "ctx");
        need(A, "A");
        need(B, "B");
        need(outs, "outs");
        for (uint32_t i = 0; i < L; i++) {
            same_ctx(ctx, A[i]);
            same_ctx(ctx, B[i]);
        }
        set_device(ctx);
        circuit_rank_blocked_finish(ctx, A, B, (int)L, outs);
        check_launch();
    });
}

rk_status rk_order_stat_blocked(rk_ctx* ctx, const rk_ct* const* blocks, uint32_t L, uint32_t k, uint32_t flags,
                                rk_ct** outs) {
    return guard([&] {
        need(ctx, "ctx");
        need(blocks, "blocks");
        need(outs, "outs");
        RK_REQUIRE(flags == RK_TIES_FIRST, RK_EINVAL, "blocked order statistic takes RK_TIES_FIRST only");
        for (uint32_t i = 0; i < L; i++) same_ctx(ctx, blocks[i]);
        set_device(ctx);
        circuit_order_stat_blocked(ctx, blocks, (int)L, k, outs);
        check_launch();
    });
}

rk_status rk_sort_blocked(rk_ctx* ctx, const rk_ct* const* blocks, uint32_t L, uint32_t flags, rk_ct** outs) {
    return guard([&] {
        need(ctx, "ctx");
        need(blocks, "blocks");
        need(outs, "outs");
        RK_REQUIRE(flags == 0, RK_EINVAL, "blocked sort takes no flags");
        for (uint32_t i = 0; i < L; i++) same_ctx(ctx, blocks[i]);
        set_device(ctx);
        circuit_sort_blocked(ctx, blocks, (int)L, outs);
        check_launch();
    });
}

rk_status rk_server_start(rk_ctx* ctx, size_t mem_budget_bytes, uint32_t max_stack) {
    return guard([&] {
        need(ctx, "ctx");
        set_device(ctx);
        server_start(ctx, mem_budget_bytes, (int)max_stack);
    });
}

rk_status rk_server_submit(rk_ctx* ctx, uint32_t op, uint32_t arg, uint32_t flags, const rk_ct* in, uint64_t* ticket) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, in);
        need(ticket, "ticket");
        *ticket = server_submit(ctx, op, arg, flags, in);
    });
}

rk_status rk_server_wait(rk_ctx* ctx, uint64_t ticket, double timeout_s, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        need(out, "out");
        *out = nullptr;
        *out = server_collect(ctx, ticket, timeout_s);
    });
}

rk_status rk_server_poll(rk_ctx* ctx, uint64_t ticket, rk_ct** out) { return rk_server_wait(ctx, ticket, 0.0, out); }

rk_status rk_server_stats(rk_ctx* ctx, double out[8]) {
    return guard([&] {
        need(ctx, "ctx");
        need(out, "out");
        server_stats(ctx, out);
    });
}

rk_status rk_server_stats_lanes(rk_ctx* ctx, double out[5]) {
    return guard([&] {
        need(ctx, "ctx");
        need(out, "out");
        server_stats_lanes(ctx, out);
    });
}

rk_status rk_server_latencies(rk_ctx* ctx, double* out, size_t cap, size_t* count) {
    return guard([&] {
        need(ctx, "ctx");
        need(count, "count");
        RK_REQUIRE(out || cap == 0, RK_EINVAL, "out is NULL");
        *count = server_latencies(ctx, out, cap);
    });
}

rk_status rk_server_stop(rk_ctx* ctx) {
    return guard([&] {
        need(ctx, "ctx");
        set_device(ctx);
        server_stop(ctx);
    });
}

rk_status rk_graph_rank(rk_ctx* ctx, const rk_ct* tmpl, uint32_t flags, rk_graph** out) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, tmpl);
        need(out, "out");
        set_device(ctx);
        *out = graph_rank_capture(ctx, tmpl, flags);
    });
}

rk_status rk_graph_capture(rk_ctx* ctx, uint32_t op, uint32_t arg, uint32_t flags, uint32_t L, const rk_ct* tmpl,
                           rk_graph** out) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, tmpl);
        need(out, "out");
        set_device(ctx);
        *out = graph_capture(ctx, op, arg, flags, (int)L, tmpl);
    });
}

rk_status rk_graph_run(rk_graph* g, const rk_ct* in, rk_ct** out) {
    return guard([&] {
        need(g, "graph");
        need(out, "out");
        rk_ctx* ctx = graph_context(g);
        same_ctx(ctx, in);
        set_device(ctx);
        *out = graph_rank_run(g, in);
    });
}

void rk_graph_free(rk_graph* g) { graph_free(g); }

rk_status rk_ct_stack(rk_ctx* ctx, const rk_ct* const* in, uint32_t count, rk_ct** out) {
    return guard([&] {
        need(ctx, "ctx");
        need(in, "in");
        need(out, "out");
        for (uint32_t i = 0; i < count; i++) same_ctx(ctx, in[i]);
        set_device(ctx);
        *out = ct_stack(ctx, in, (int)count);
    });
}

rk_status rk_ct_unstack(rk_ctx* ctx, const rk_ct* in, rk_ct** outs) {
    return guard([&] {
        need(ctx, "ctx");
        same_ctx(ctx, in);
        need(outs, "outs");
        set_device(ctx);
        ct_unstack(ctx, in, outs);
    });
}

uint32_t rk_ct_count(const rk_ct* ct) { return ct ? (uint32_t)ct->B : 0; }

rk_status rk_rescale_noalloc(rk_ctx* ctx, const uint64_t* d_in, uint64_t* d_out, uint32_t level) {
    return guard([&] {
        need(ctx, "ctx");
        rescale_noalloc(ctx, (const u64*)d_in, (u64*)d_out, (int)level);
    });
}

rk_status rk_profile_start(rk_ctx* ctx, const char* kinds) {
    return guard([&] {
        need(ctx, "ctx");
        Profiler& p = ctx->prof;
        p.mask = 0;
        p.used = 0;
        p.paused = false;
        for (int k = 0; k < KK_COUNT; k++) {
            p.bytes[k] = p.ops[k] = p.ms[k] = 0;
            p.timed[k] = 0;
        }
        if (!kinds || !kinds[0]) return;
        uint32_t mask = 0;
        std::string list(kinds);
        size_t at = 0;
        while (at <= list.size()) {
            const size_t end = std::min(list.find(',', at), list.size());
            const std::string name = list.substr(at, end - at);
            int found = -1;
            for (int k = 0; k < KK_COUNT; k++)
                if (name == kKernelKindNames[k]) found = k;
            RK_REQUIRE(found >= 0, RK_EINVAL, "unknown kernel kind " + name);
            mask |= 1u << found;
            at = end + 1;
        }
        p.mask = mask;
    });
}

rk_status rk_profile_stop(rk_ctx* ctx, double out[4]) {
    return guard([&] {
        need(ctx, "ctx");
        need(out, "out");
        set_device(ctx);
        Profiler& p = ctx->prof;
        RK_CUDA(cudaStreamSynchronize(ctx->stream));
        for (size_t i = 0; i + 1 < p.used; i += 2) {
            float t = 0;
            RK_CUDA(cudaEventElapsedTime(&t, p.ev[i], p.ev[i + 1]));
            p.ms[p.ev_kind[i]] += t;
        }
        out[0] = out[1] = out[2] = out[3] = 0;
        for (int k = 0; k < KK_COUNT; k++) {
            out[0] += p.ms[k];
            out[1] += (double)p.timed[k];
            out[2] += p.bytes[k];
            out[3] += p.ops[k];
        }
        p.mask = 0;
        p.used = 0;
    });
}

rk_status rk_profile_pause(rk_ctx* ctx, int paused) {
    return guard([&] {
        need(ctx, "ctx");
        ctx->prof.paused = paused != 0;
    });
}

rk_status rk_profile_kind(const rk_ctx* ctx, const char* kind, double out[4]) {
    return guard([&] {
        need(ctx, "ctx");
        need(kind, "kind");
        need(out, "out");
        int found = -1;
        for (int k = 0; k < KK_COUNT; k++)
            if (std::strcmp(kind, kKernelKindNames[k]) == 0) found = k;
        RK_REQUIRE(found >= 0, RK_EINVAL, std::string("unknown kernel kind ") + kind);
        const Profiler& p = ctx->prof;
        out[0] = p.ms[found];
        out[1] = (double)p.timed[found];
        out[2] = p.bytes[found];
        out[3] = p.ops[found];
    });
}

uint64_t rk_launch_count(const rk_ctx* ctx) { return ctx ? ctx->prof.launches : 0; }

rk_status rk_ntt_forward(rk_ctx* ctx, uint64_t* d_data, uint32_t limbs, uint32_t first_prime) {
    return guard([&] {
        need(ctx, "ctx");
        need(d_data, "d_data");
        RK_REQUIRE(first_prime + limbs <= (uint32_t)ctx->n_primes, RK_EINVAL, "prime range out of bounds");
        set_device(ctx);
        launch_ntt_forward(ctx->env, LimbSet{(u64*)d_data, 0, 1, (int)limbs, (int)limbs, (int)first_prime, 0}, ctx->stream);
        check_launch();
    });
}

rk_status rk_ntt_inverse(rk_ctx* ctx, uint64_t* d_data, uint32_t limbs, uint32_t first_prime) {
    return guard([&] {
        need(ctx, "ctx");
        need(d_data, "d_data");
        RK_REQUIRE(first_prime + limbs <= (uint32_t)ctx->n_primes, RK_EINVAL, "prime range out of bounds");
        set_device(ctx);
        launch_ntt_inverse(ctx->env, LimbSet{(u64*)d_data, 0, 1, (int)limbs, (int)limbs, (int)first_prime, 0}, ctx->stream);
        check_launch();
    });
}

}  // extern "C"
