// CUDA-graph capture of a whole circuit for one input shape: the rank (Alg. 3 /
// Alg. 6), the order statistic (Alg. 4), the sort (Alg. 5) and their blocked forms
// (Alg. 7, Alg. 8), on single or stacked ciphertexts.
//
// A circuit's host logic is static for a given (operation, arguments, level, N, Q,
// n_real, stack size): rotation amounts, levels and constants do not depend on the
// data.  So the circuit is run once to build every cached plaintext and size the
// scratch, then captured on the context stream; its stream-ordered allocations
// become graph memory nodes.  A replay copies the new input into the captured input
// buffer, launches the graph and copies the result out.
#include "kernels.cuh"

rk_ct* circuit_rank(rk_ctx* c, const rk_ct* in, uint32_t flags);
rk_ct* circuit_order_stat(rk_ctx* c, const rk_ct* in, uint32_t k, uint32_t flags);
rk_ct* circuit_sort(rk_ctx* c, const rk_ct* in, uint32_t flags);
void circuit_rank_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs);
void circuit_rank_blocked_tc(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs);
void circuit_order_stat_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, uint32_t k, rk_ct** outs);
void circuit_sort_blocked(rk_ctx* c, const rk_ct* const* blocks, int L, rk_ct** outs);

struct rk_graph {
    rk_ctx* ctx = nullptr;
    rk_ct* input = nullptr;           // captured input buffer
    std::vector<rk_ct> out_meta;      // shape, level and device address of each captured output
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool launched = false;
    uint32_t op = RK_OP_RANK, arg = 0, flags = 0;
    int L = 1;                        // blocks of a blocked operation
    uint64_t kernels = 0;             // kernel nodes in the graph
    uint64_t generation = 0;          // context generation the graph's pointers belong to
};

namespace {

// The circuit of `g` on `in`: one output, or (blocked operations) the L output blocks,
// in[i] being members [i Bq, (i+1) Bq) of the stacked input.
std::vector<rk_ct*> run_circuit(rk_ctx* c, const rk_graph* g, const rk_ct* in) {
    if (g->op < RK_OP_RANK_BLOCKED) {
        rk_ct* y = nullptr;
        if (g->op == RK_OP_RANK) y = circuit_rank(c, in, g->flags);
        else if (g->op == RK_OP_ORDER_STAT) y = circuit_order_stat(c, in, g->arg, g->flags);
        else y = circuit_sort(c, in, g->flags);
        return {y};
    }
    const int L = g->L, Bq = in->B / L;
    std::vector<rk_ct*> views(L, nullptr), outs(L, nullptr);
    try {
        for (int i = 0; i < L; i++) views[i] = ct_view_range(in, i * Bq, Bq);
        if (g->op == RK_OP_RANK_BLOCKED && (g->flags & RK_TIES_CORRECT))
            circuit_rank_blocked_tc(c, views.data(), L, outs.data());
        else if (g->op == RK_OP_RANK_BLOCKED)
            circuit_rank_blocked(c, views.data(), L, outs.data());
        else if (g->op == RK_OP_ORDER_STAT_BLOCKED)
            circuit_order_stat_blocked(c, views.data(), L, g->arg, outs.data());
        else
            circuit_sort_blocked(c, views.data(), L, outs.data());
    } catch (...) {
        for (auto* v : views) ct_free(v);
        for (auto* o : outs) ct_free(o);
        throw;
    }
    for (auto* v : views) ct_free(v);
    return outs;
}

}  // namespace

rk_graph* graph_capture(rk_ctx* c, uint32_t op, uint32_t arg, uint32_t flags, int L, const rk_ct* tmpl) {
    RK_REQUIRE(op >= RK_OP_RANK && op <= RK_OP_SORT_BLOCKED, RK_EINVAL, "unknown circuit for a graph");
    RK_REQUIRE(op >= RK_OP_RANK_BLOCKED ? (L >= 1 && tmpl->B % L == 0) : L == 1, RK_EINVAL,
               "a blocked graph takes a stack of L blocks (L dividing the stack size); other circuits L = 1");
    RK_REQUIRE(!c->server, RK_EINVAL, "graph capture while a server runs");
    rk_graph* g = new rk_graph();
    g->ctx = c;
    g->op = op;
    g->arg = arg;
    g->flags = flags;
    g->L = L;
    try {
        // warm-up: plaintext caches and scratch sized for this stack
        for (auto* w : run_circuit(c, g, tmpl)) ct_free(w);
        RK_CUDA(cudaStreamSynchronize(c->stream));
        g->generation = c->generation;
        g->input = ct_clone_meta(tmpl, tmpl->level);
        ev_copy(c, tmpl, g->input);
        RK_CUDA(cudaStreamSynchronize(c->stream));
    } catch (...) {
        ct_free(g->input);
        delete g;
        throw;
    }
    const uint32_t saved = c->prof.mask;
    const uint64_t launches = c->prof.launches;   // captured kernels run only on replay
    c->prof.mask = 0;
    RK_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    std::vector<rk_ct*> outs;
    try {
        outs = run_circuit(c, g, g->input);
    } catch (...) {
        cudaGraph_t dummy = nullptr;
        cudaStreamEndCapture(c->stream, &dummy);
        if (dummy) cudaGraphDestroy(dummy);
        c->prof.mask = saved;
        c->prof.launches = launches;
        ct_free(g->input);
        delete g;
        throw;
    }
    cudaError_t e = cudaStreamEndCapture(c->stream, &g->graph);
    c->prof.mask = saved;
    c->prof.launches = launches;
    for (auto* o : outs) {
        rk_ct m = *o;
        m.view = true;           // the graph owns this address
        g->out_meta.push_back(m);
        o->view = true;
        ct_free(o);
    }
    if (e != cudaSuccess) {
        ct_free(g->input);
        delete g;
        throw rk_error(RK_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    }
    size_t nodes = 0;
    cudaGraphGetNodes(g->graph, nullptr, &nodes);
    std::vector<cudaGraphNode_t> list(nodes);
    cudaGraphGetNodes(g->graph, list.data(), &nodes);
    for (auto nd : list) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) g->kernels++;
    }
    e = cudaGraphInstantiateWithFlags(&g->exec, g->graph, cudaGraphInstantiateFlagAutoFreeOnLaunch);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g->graph);
        ct_free(g->input);
        delete g;
        throw rk_error(RK_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    }
    return g;
}

rk_graph* graph_rank_capture(rk_ctx* c, const rk_ct* tmpl, uint32_t flags) {
    return graph_capture(c, RK_OP_RANK, 0, flags, 1, tmpl);
}

// Replay on `in` (shaped like the template): one output handle; for a blocked
// circuit, the stack of its L output blocks (block-major, Bq members each).
rk_ct* graph_rank_run(rk_graph* g, const rk_ct* in) {
    rk_ctx* c = g->ctx;
    const rk_ct* t = g->input;
    RK_REQUIRE(in->level == t->level && in->B == t->B && in->N == t->N && in->Q == t->Q && in->n_real == t->n_real &&
                   in->layout == t->layout,
               RK_EINVAL, "input shape differs from the captured one");
    RK_REQUIRE(g->generation == c->generation, RK_EINVAL,
               "the context changed since the capture (scratch grown, keys, masks or indicator replaced): capture again");
    ev_copy(c, in, g->input);
    RK_CUDA(cudaGraphLaunch(g->exec, c->stream));
    g->launched = true;
    c->prof.launches += g->kernels;
    if (g->out_meta.size() == 1) {
        rk_ct* out = ct_clone_meta(&g->out_meta[0], g->out_meta[0].level);
        out->view = false;
        ev_copy(c, &g->out_meta[0], out);
        return out;
    }
    std::vector<const rk_ct*> parts;
    for (auto& m : g->out_meta) parts.push_back(&m);
    return ct_stack(c, parts.data(), (int)parts.size());
}

void graph_free(rk_graph* g) {
    if (!g) return;
    rk_ctx* c = g->ctx;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (g->launched)   // the last launch's allocations
        for (auto& m : g->out_meta) cudaFreeAsync(m.data, c->stream);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    ct_free(g->input);
    cudaStreamSynchronize(c->stream);
    delete g;
}

rk_ctx* graph_context(const rk_graph* g) { return g->ctx; }
