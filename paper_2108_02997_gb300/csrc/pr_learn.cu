// pr_learn.cu — learned warm start: features, MLP inference and training.
// (Filled in below; entry points exist so the ABI is complete.)
#include "pr_internal.cuh"

struct pr_mlp {
    uint32_t magic;
};

bool pr_mlp_valid(const pr_mlp *m) { return m && registry_has(m) && m->magic == kMlpMagic; }

pr_status pr_learned_start(const pr_mlp *, const pr_graph *, double, double *, cudaStream_t) {
    return pr_fail(PR_ENOTSUP, "learned warm start not available in this build");
}

extern "C" pr_status pr_mlp_create(const float *, pr_mlp **out) {
    if (out) *out = nullptr;
    return pr_fail(PR_ENOTSUP, "learned warm start not available in this build");
}
extern "C" pr_status pr_mlp_destroy(pr_mlp *) { return PR_OK; }
extern "C" pr_status pr_mlp_get_params(const pr_mlp *, float *) {
    return pr_fail(PR_ENOTSUP, "learned warm start not available in this build");
}
extern "C" pr_status pr_features(const pr_graph *, double, float *, void *) {
    return pr_fail(PR_ENOTSUP, "learned warm start not available in this build");
}
extern "C" pr_status pr_mlp_warm_start(const pr_mlp *, const pr_graph *, double, double *, void *) {
    return pr_fail(PR_ENOTSUP, "learned warm start not available in this build");
}
extern "C" pr_status pr_mlp_train(pr_mlp *, const pr_graph *const *, const double *, const double *const *, int32_t,
                                  int32_t, float, float *, void *) {
    return pr_fail(PR_ENOTSUP, "learned warm start not available in this build");
}
