// A trained stop network as a C caller holds it: parameters and feature
// standardisation copied into one caller-owned device buffer, the output
// scaling and acceptance rules in the rbf_stopnet host fields, and a small
// binary file format to save and load all of it (no Python needed to run the
// learned stop from C).
//
// File layout (native little-endian, as on every platform the library builds
// for): 8-byte magic "RBFSTOP1"; int32 n_in, n_hidden, n_out, n_params,
// feat_steps; float params[n_params], feat_mean[n_in], feat_std[n_in],
// out_mean[2], out_std[2]; int32 l_min, l_max, window, fallback_rule;
// float64 accept_tol, t_min, t_max, z_max.
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.h"

namespace {

constexpr char MAGIC[8] = {'R', 'B', 'F', 'S', 'T', 'O', 'P', '1'};

rbf_status check_rules(rbf_ctx* ctx, int l_min, int l_max, int window, int fallback_rule, int feat_steps) {
    if (feat_steps < 1 || feat_steps > 10)
        return rbf_fail(ctx, RBF_ERR_INVALID, "stop network: feat_steps %d outside [1, 10]", feat_steps);
    if (l_min < feat_steps || l_max < l_min || l_max > 1023)
        return rbf_fail(ctx, RBF_ERR_INVALID, "stop network: need feat_steps <= l_min <= l_max <= 1023");
    if (window < 0) return rbf_fail(ctx, RBF_ERR_INVALID, "stop network: negative window");
    if (fallback_rule != RBF_GCV && fallback_rule != RBF_LCURVE)
        return rbf_fail(ctx, RBF_ERR_INVALID, "stop network: fallback rule must be RBF_GCV or RBF_LCURVE");
    return RBF_OK;
}

}  // namespace

extern "C" rbf_status rbf_stopnet_init(rbf_ctx* ctx, rbf_stopnet* net, float* d_storage, const float* h_params,
                                       const float* h_feat_mean, const float* h_feat_std, const float* h_out,
                                       const int* h_rules, const double* h_tols) {
    RbfRange range_("rbf_stopnet_init");
    if (!ctx) return RBF_ERR_INVALID;
    if (!net || !d_storage || !h_params || !h_out || !h_rules || !h_tols)
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_stopnet_init: NULL argument");
    if ((h_feat_mean == nullptr) != (h_feat_std == nullptr))
        return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_stopnet_init: give both feature mean and std, or neither");
    RBF_TRY(check_rules(ctx, h_rules[0], h_rules[1], h_rules[2], h_rules[3], 10));
    for (int i = 0; i < 2; ++i)
        if (!(h_out[2 + i] > 0.0f)) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_stopnet_init: output std must be > 0");
    std::vector<float> buf(RBF_STOPNET_DEVICE_FLOATS, 0.0f);
    std::memcpy(buf.data(), h_params, sizeof(float) * RBF_MLP_PARAMS);
    if (h_feat_mean) {
        std::memcpy(buf.data() + RBF_MLP_PARAMS, h_feat_mean, sizeof(float) * RBF_MLP_IN);
        std::memcpy(buf.data() + RBF_MLP_PARAMS + RBF_MLP_IN, h_feat_std, sizeof(float) * RBF_MLP_IN);
    }
    RBF_CUDA(ctx, cudaMemcpyAsync(d_storage, buf.data(), sizeof(float) * buf.size(), cudaMemcpyHostToDevice,
                                  ctx->stream));
    RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));  // buf is a host temporary
    net->d_params = d_storage;
    net->d_feat_mean = h_feat_mean ? d_storage + RBF_MLP_PARAMS : nullptr;
    net->d_feat_std = h_feat_mean ? d_storage + RBF_MLP_PARAMS + RBF_MLP_IN : nullptr;
    net->out_mean[0] = h_out[0];
    net->out_mean[1] = h_out[1];
    net->out_std[0] = h_out[2];
    net->out_std[1] = h_out[3];
    net->feat_steps = 10;
    net->l_min = h_rules[0];
    net->l_max = h_rules[1];
    net->window = h_rules[2];
    net->fallback_rule = h_rules[3];
    net->accept_tol = h_tols[0];
    net->t_min = h_tols[1];
    net->t_max = h_tols[2];
    net->z_max = h_tols[3];
    return RBF_OK;
}

extern "C" rbf_status rbf_stopnet_save(rbf_ctx* ctx, const rbf_stopnet* net, const char* path) {
    RbfRange range_("rbf_stopnet_save");
    if (!ctx) return RBF_ERR_INVALID;
    if (!net || !net->d_params || !path) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_stopnet_save: NULL argument");
    std::vector<float> p(RBF_MLP_PARAMS), mean(RBF_MLP_IN, 0.0f), sd(RBF_MLP_IN, 1.0f);
    RBF_CUDA(ctx, cudaMemcpyAsync(p.data(), net->d_params, sizeof(float) * p.size(), cudaMemcpyDeviceToHost,
                                  ctx->stream));
    if (net->d_feat_mean && net->d_feat_std) {
        RBF_CUDA(ctx, cudaMemcpyAsync(mean.data(), net->d_feat_mean, sizeof(float) * RBF_MLP_IN,
                                      cudaMemcpyDeviceToHost, ctx->stream));
        RBF_CUDA(ctx, cudaMemcpyAsync(sd.data(), net->d_feat_std, sizeof(float) * RBF_MLP_IN, cudaMemcpyDeviceToHost,
                                      ctx->stream));
    }
    RBF_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_stopnet_save: cannot open %s", path);
    const int32_t dims[5] = {RBF_MLP_IN, RBF_MLP_HIDDEN, RBF_MLP_OUT, RBF_MLP_PARAMS, net->feat_steps};
    const float outs[4] = {net->out_mean[0], net->out_mean[1], net->out_std[0], net->out_std[1]};
    const int32_t rules[4] = {net->l_min, net->l_max, net->window, net->fallback_rule};
    const double tols[4] = {net->accept_tol, net->t_min, net->t_max, net->z_max};
    bool ok = std::fwrite(MAGIC, 1, 8, fp) == 8 && std::fwrite(dims, sizeof(dims), 1, fp) == 1 &&
              std::fwrite(p.data(), sizeof(float), p.size(), fp) == p.size() &&
              std::fwrite(mean.data(), sizeof(float), mean.size(), fp) == mean.size() &&
              std::fwrite(sd.data(), sizeof(float), sd.size(), fp) == sd.size() &&
              std::fwrite(outs, sizeof(outs), 1, fp) == 1 && std::fwrite(rules, sizeof(rules), 1, fp) == 1 &&
              std::fwrite(tols, sizeof(tols), 1, fp) == 1;
    ok = (std::fclose(fp) == 0) && ok;
    if (!ok) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_stopnet_save: writing %s failed", path);
    return RBF_OK;
}

extern "C" rbf_status rbf_stopnet_load(rbf_ctx* ctx, const char* path, rbf_stopnet* net, float* d_storage) {
    RbfRange range_("rbf_stopnet_load");
    if (!ctx) return RBF_ERR_INVALID;
    if (!path || !net || !d_storage) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_stopnet_load: NULL argument");
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_stopnet_load: cannot open %s", path);
    char magic[8];
    int32_t dims[5];
    std::vector<float> p(RBF_MLP_PARAMS), mean(RBF_MLP_IN), sd(RBF_MLP_IN);
    float outs[4];
    int32_t rules[4];
    double tols[4];
    bool ok = std::fread(magic, 1, 8, fp) == 8 && std::memcmp(magic, MAGIC, 8) == 0 &&
              std::fread(dims, sizeof(dims), 1, fp) == 1 && dims[0] == RBF_MLP_IN && dims[1] == RBF_MLP_HIDDEN &&
              dims[2] == RBF_MLP_OUT && dims[3] == RBF_MLP_PARAMS &&
              std::fread(p.data(), sizeof(float), p.size(), fp) == p.size() &&
              std::fread(mean.data(), sizeof(float), mean.size(), fp) == mean.size() &&
              std::fread(sd.data(), sizeof(float), sd.size(), fp) == sd.size() &&
              std::fread(outs, sizeof(outs), 1, fp) == 1 && std::fread(rules, sizeof(rules), 1, fp) == 1 &&
              std::fread(tols, sizeof(tols), 1, fp) == 1;
    char extra;
    ok = ok && std::fread(&extra, 1, 1, fp) == 0;  // nothing after the last field
    std::fclose(fp);
    if (!ok) return rbf_fail(ctx, RBF_ERR_INVALID, "rbf_stopnet_load: %s is not a stop-network file of this layout",
                             path);
    RBF_TRY(check_rules(ctx, rules[0], rules[1], rules[2], rules[3], dims[4]));
    const int ri[4] = {rules[0], rules[1], rules[2], rules[3]};
    RBF_TRY(rbf_stopnet_init(ctx, net, d_storage, p.data(), mean.data(), sd.data(), outs, ri, tols));
    net->feat_steps = dims[4];
    return RBF_OK;
}
