// C ABI of the learned channel-estimate denoiser (pusch_cnn_*, pusch_ls_grid, pusch_chest_cnn).
#include <stdio.h>

#include "internal.cuh"

namespace {

pusch_status cfail(pusch_status st, const char *msg, cudaError_t e = cudaSuccess) {
    char buf[512];
    if (e != cudaSuccess)
        snprintf(buf, sizeof buf, "%s: %s", msg, cudaGetErrorString(e));
    else
        snprintf(buf, sizeof buf, "%s", msg);
    pusch::set_last_error(buf);
    return st;
}

pusch_status grid_check(int n, int w) {
    if (n < 0 || n > 65535) return cfail(PUSCH_ERR_ARG, "number of grids must be in [0, 65535]");
    if (w < 1 || w > 1 << 20) return cfail(PUSCH_ERR_ARG, "grid width must be in [1, 2^20]");
    return PUSCH_OK;
}

}  // namespace

extern "C" {

int pusch_cnn_param_count(void) { return pusch::cnn_param_count(); }

pusch_status pusch_cnn_forward(int n, int w, const void *x, const void *params, float *y, void *acts, void *stream) {
    pusch_status st = grid_check(n, w);
    if (st != PUSCH_OK) return st;
    if (n == 0) return PUSCH_OK;
    if (!x || !params || !y || !acts) return cfail(PUSCH_ERR_ARG, "pusch_cnn_forward: NULL buffer");
    cudaError_t e = pusch::cnn_forward(n, w, (const __nv_bfloat16 *)x, (const __nv_bfloat16 *)params, y,
                                       (__nv_bfloat16 *)acts, (cudaStream_t)stream);
    if (e != cudaSuccess) return cfail(PUSCH_ERR_CUDA, "CNN forward launch", e);
    pusch::set_last_error("");
    return PUSCH_OK;
}

pusch_status pusch_cnn_backward(int n, int w, const void *x, const void *acts, const void *params, const float *y,
                                const float *target, float *grad, float *loss, float *work, void *wflip,
                                void *stream) {
    pusch_status st = grid_check(n, w);
    if (st != PUSCH_OK) return st;
    if (n == 0) return PUSCH_OK;
    if (!x || !acts || !params || !y || !target || !grad || !work || !wflip)
        return cfail(PUSCH_ERR_ARG, "pusch_cnn_backward: NULL buffer");
    cudaError_t e = pusch::cnn_backward(n, w, (const __nv_bfloat16 *)x, (const __nv_bfloat16 *)acts,
                                        (const __nv_bfloat16 *)params, y, target, grad, loss, work,
                                        (__nv_bfloat16 *)wflip, (cudaStream_t)stream);
    if (e != cudaSuccess) return cfail(PUSCH_ERR_CUDA, "CNN backward launch", e);
    pusch::set_last_error("");
    return PUSCH_OK;
}

pusch_status pusch_cnn_adam(int step, float lr, float beta1, float beta2, float eps, float *params, void *params_bf16,
                            const float *grad, float *m, float *v, void *stream) {
    if (step < 1) return cfail(PUSCH_ERR_ARG, "Adam step counts from 1");
    if (!params || !params_bf16 || !grad || !m || !v) return cfail(PUSCH_ERR_ARG, "pusch_cnn_adam: NULL buffer");
    cudaError_t e = pusch::cnn_adam(step, lr, beta1, beta2, eps, params, (__nv_bfloat16 *)params_bf16, grad, m, v,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cfail(PUSCH_ERR_CUDA, "Adam launch", e);
    pusch::set_last_error("");
    return PUSCH_OK;
}

pusch_status pusch_ls_grid(pusch_handle *h, int n_slots, const void *beam, const void *pilots, void *grid, float *scale,
                           void *stream) {
    if (!h) return cfail(PUSCH_ERR_ARG, "handle is NULL");
    if (n_slots < 0 || n_slots > h->max_slots) return cfail(PUSCH_ERR_ARG, "n_slots out of [0, max_slots]");
    if (n_slots == 0) return PUSCH_OK;
    if (!beam || !pilots || !grid || !scale) return cfail(PUSCH_ERR_ARG, "pusch_ls_grid: NULL buffer");
    if (h->geo.dmrs_type != 0) return cfail(PUSCH_ERR_UNSUPPORTED, "the learned estimator uses the comb pilot model");
    cudaError_t e = pusch::launch_ls_grid(h->geo, n_slots, (const float2 *)beam, (const float2 *)pilots,
                                          (__nv_bfloat16 *)grid, scale, (cudaStream_t)stream);
    if (e != cudaSuccess) return cfail(PUSCH_ERR_CUDA, "LS grid launch", e);
    pusch::set_last_error("");
    return PUSCH_OK;
}

pusch_status pusch_chest_cnn(pusch_handle *h, int n_slots, const void *beam, const void *pilots, const void *params,
                             float kappa, void *H_hat, float *resid, uint8_t *fallback, void *stream) {
    if (!h) return cfail(PUSCH_ERR_ARG, "handle is NULL");
    if (n_slots < 0 || n_slots > h->max_slots) return cfail(PUSCH_ERR_ARG, "n_slots out of [0, max_slots]");
    if (n_slots == 0) return PUSCH_OK;
    if (!beam || !pilots || !params || !H_hat) return cfail(PUSCH_ERR_ARG, "pusch_chest_cnn: NULL buffer");
    if (!(kappa > 0.f)) return cfail(PUSCH_ERR_ARG, "kappa must be > 0");
    if (h->geo.dmrs_type != 0) return cfail(PUSCH_ERR_UNSUPPORTED, "the learned estimator uses the comb pilot model");
    const pusch::Geometry &g = h->geo;
    const long long grids_max = (long long)h->max_slots * g.n_layers * g.n_beams;
    if (grids_max > 65535) return cfail(PUSCH_ERR_UNSUPPORTED, "max_slots * n_layers * n_beams exceeds 65535 grids");
    cudaError_t e;
    if (!h->cnn_grid) {  // workspace sized for max_slots, allocated on first use
        const size_t px = (size_t)grids_max * 2 * g.n_sc;
        if ((e = cudaMalloc(&h->cnn_grid, px * 2 * sizeof(__nv_bfloat16))) != cudaSuccess ||
            (e = cudaMalloc((void **)&h->cnn_scale, (size_t)grids_max * sizeof(float))) != cudaSuccess ||
            (e = cudaMalloc(&h->cnn_acts, (size_t)grids_max * 2 * ((g.n_sc + 7) & ~7) * 3 * 32 * sizeof(__nv_bfloat16))) !=
                cudaSuccess ||
            (e = cudaMalloc((void **)&h->cnn_y, px * 2 * sizeof(float))) != cudaSuccess)
            return cfail(PUSCH_ERR_CUDA, "CNN workspace allocation", e);
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int grids = n_slots * g.n_layers * g.n_beams;
    if ((e = pusch::launch_chest_ls(g, n_slots, (const float2 *)beam, (const float2 *)pilots, (float2 *)H_hat, h->ls,
                                    s)) !=
        cudaSuccess)
        return cfail(PUSCH_ERR_CUDA, "plain LS launch", e);
    if ((e = pusch::launch_ls_grid(g, n_slots, (const float2 *)beam, (const float2 *)pilots,
                                   (__nv_bfloat16 *)h->cnn_grid, h->cnn_scale, s)) != cudaSuccess)
        return cfail(PUSCH_ERR_CUDA, "LS grid launch", e);
    // activation rows padded to a multiple of 8 subcarriers, so that the 32 -> 32 layers run on the tensor cores
    if ((e = pusch::cnn_forward(grids, g.n_sc, (const __nv_bfloat16 *)h->cnn_grid, (const __nv_bfloat16 *)params,
                                h->cnn_y, (__nv_bfloat16 *)h->cnn_acts, s, (g.n_sc + 7) & ~7, h->kernel_err)) !=
        cudaSuccess)
        return cfail(PUSCH_ERR_CUDA, "CNN forward launch", e);
    if ((e = pusch::launch_cnn_to_h(g, n_slots, kappa, h->cnn_y, h->cnn_scale, (const float2 *)beam,
                                    (const float2 *)pilots, (float2 *)H_hat, resid, fallback, s)) != cudaSuccess)
        return cfail(PUSCH_ERR_CUDA, "CNN estimate launch", e);
    pusch::set_last_error("");
    return PUSCH_OK;
}

}  // extern "C"
