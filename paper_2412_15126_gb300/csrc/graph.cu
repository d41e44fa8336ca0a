// CUDA-graph capture of a whole rank circuit (Alg. 3 / Alg. 6) for one input shape.
//
// The circuit's host logic is static for a given (level, N, Q, n_real, stack size,
// flags): rotation amounts, levels and constants do not depend on the data.  So the
// circuit is run once to build every cached plaintext and size the scratch, then
// captured on the context stream; its stream-ordered allocations become graph
// memory nodes.  A replay copies the new input into the captured input buffer,
// launches the graph and copies the result out.
#include "kernels.cuh"

rk_ct* circuit_rank(rk_ctx* c, const rk_ct* in, uint32_t flags);

struct rk_graph {
    rk_ctx* ctx = nullptr;
    rk_ct* input = nullptr;     // captured input buffer
    rk_ct out_meta{};           // shape, level and device address of the captured output
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool launched = false;
    uint32_t flags = 0;
    uint64_t kernels = 0;       // kernel nodes in the graph
    uint64_t generation = 0;    // context generation the graph's pointers belong to
};

rk_graph* graph_rank_capture(rk_ctx* c, const rk_ct* tmpl, uint32_t flags) {
    // warm-up: plaintext caches and scratch sized for this stack
    rk_ct* w = circuit_rank(c, tmpl, flags);
    ct_free(w);
    RK_CUDA(cudaStreamSynchronize(c->stream));
    rk_graph* g = new rk_graph();
    g->ctx = c;
    g->flags = flags;
    g->generation = c->generation;
    g->input = ct_clone_meta(tmpl, tmpl->level);
    ev_copy(c, tmpl, g->input);
    RK_CUDA(cudaStreamSynchronize(c->stream));
    const uint32_t saved = c->prof.mask;
    const uint64_t launches = c->prof.launches;   // captured kernels run only on replay
    c->prof.mask = 0;
    RK_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    rk_ct* out = nullptr;
    try {
        out = circuit_rank(c, g->input, flags);
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
    g->out_meta = *out;
    g->out_meta.view = true;     // the graph owns this address
    out->view = true;
    ct_free(out);
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
    rk_ct* out = ct_clone_meta(&g->out_meta, g->out_meta.level);
    out->view = false;
    ev_copy(c, &g->out_meta, out);
    c->prof.launches += g->kernels;
    return out;
}

void graph_free(rk_graph* g) {
    if (!g) return;
    rk_ctx* c = g->ctx;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    if (g->launched) cudaFreeAsync(g->out_meta.data, c->stream);   // last launch's allocation
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    ct_free(g->input);
    cudaStreamSynchronize(c->stream);
    delete g;
}

rk_ctx* graph_context(const rk_graph* g) { return g->ctx; }
