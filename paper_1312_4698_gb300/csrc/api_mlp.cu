// C-ABI entry points of the learned residual (declared in include/scivr_mlp.h):
// weight upload and tiling, batched evaluation, the training objective's
// gradient, AdamW, and the analytic FP64 evaluation that checks them.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "scivr_internal.cuh"

using namespace scivr;

namespace {

int err(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(code, buf);
}

int64_t n_params(int F, int H) { return (int64_t)H * F + 2LL * H * H + 4LL * H + 1; }

bool finite_n(const double *x, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(x[i])) return false;
    return true;
}

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

int need_mlp(scivr_pes pes, const char *fn)
{
    if (!pes) return err(SCIVR_EINVAL, "%s: NULL potential", fn);
    if (pes->dev.mlp.H == 0) return err(SCIVR_EINVAL, "%s: no learned residual attached (scivr_pes_set_mlp)", fn);
    return SCIVR_OK;
}

// Point the weight record into one device block: theta | s_in | 4 BF16 tiles.
void layout(MlpWeightsDev &w, char *blob, int F, int H)
{
    const int64_t np = n_params(F, H);
    float *th = reinterpret_cast<float *>(blob);
    w.H = H;
    w.n_params = np;
    w.theta = th;
    w.W1 = th;
    w.b1 = w.W1 + (size_t)H * F;
    w.W2 = w.b1 + H;
    w.b2 = w.W2 + (size_t)H * H;
    w.W3 = w.b2 + H;
    w.b3 = w.W3 + (size_t)H * H;
    w.w4 = w.b3 + H;
    w.b4 = w.w4 + H;
    char *p = blob + a256((size_t)np * 4);
    w.s_in = reinterpret_cast<const float *>(p);
    p += 256;
    const size_t tile = (size_t)H * H * 2;
    w.W2t = reinterpret_cast<uint8_t *>(p);
    w.W3t = w.W2t + tile;
    w.W2Tt = w.W3t + tile;
    w.W3Tt = w.W2Tt + tile;
}

size_t blob_bytes(int F, int H) { return a256((size_t)n_params(F, H) * 4) + 256 + 4 * (size_t)H * H * 2; }

}  // namespace

extern "C" {

int64_t scivr_mlp_param_count(int32_t F, int32_t H)
{
    if (F < 1 || H < 1) return 0;
    return n_params(F, H);
}

int scivr_pes_set_mlp(scivr_pes pes, const scivr_mlp_desc *m)
{
    if (!pes) return err(SCIVR_EINVAL, "scivr_pes_set_mlp: NULL potential");
    const int F = pes->dev.F;
    cudaError_t e;
    if (m) {
        if (F > 9) return err(SCIVR_EUNSUPPORTED, "scivr_pes_set_mlp: F=%d > 9 not built", F);
        if (pes->dev.kind == SCIVR_PES_CART3)
            return err(SCIVR_EUNSUPPORTED, "scivr_pes_set_mlp: a learned residual needs a polynomial surface");
        if (m->H != SCIVR_MLP_HIDDEN) return err(SCIVR_EINVAL, "scivr_pes_set_mlp: H=%d (only %d built)", m->H, SCIVR_MLP_HIDDEN);
        const int H = m->H;
        if (!m->s_in || !m->W1 || !m->b1 || !m->W2 || !m->b2 || !m->W3 || !m->b3 || !m->w4)
            return err(SCIVR_EINVAL, "scivr_pes_set_mlp: NULL array");
        for (int i = 0; i < F; ++i)
            if (!(m->s_in[i] > 0.0) || !std::isfinite(m->s_in[i]))
                return err(SCIVR_EINVAL, "scivr_pes_set_mlp: s_in must be positive");
        if (!(m->s_out > 0.0) || !std::isfinite(m->s_out)) return err(SCIVR_EINVAL, "scivr_pes_set_mlp: s_out must be positive");
        if (!finite_n(m->W1, (size_t)H * F) || !finite_n(m->b1, H) || !finite_n(m->W2, (size_t)H * H) ||
            !finite_n(m->b2, H) || !finite_n(m->W3, (size_t)H * H) || !finite_n(m->b3, H) || !finite_n(m->w4, H) ||
            !std::isfinite(m->b4))
            return err(SCIVR_EINVAL, "scivr_pes_set_mlp: non-finite weight");
        std::vector<float> th;
        th.reserve((size_t)n_params(F, H));
        auto put = [&](const double *x, size_t n) { for (size_t i = 0; i < n; ++i) th.push_back((float)x[i]); };
        put(m->W1, (size_t)H * F);
        put(m->b1, H);
        put(m->W2, (size_t)H * H);
        put(m->b2, H);
        put(m->W3, (size_t)H * H);
        put(m->b3, H);
        put(m->w4, H);
        th.push_back((float)m->b4);
        std::vector<float> sin(64, 0.0f);
        for (int i = 0; i < F; ++i) sin[i] = (float)m->s_in[i];
        void *blob = nullptr;
        e = cudaMalloc(&blob, blob_bytes(F, H));
        if (e != cudaSuccess) return cuda_error(e, "scivr_pes_set_mlp: cudaMalloc");
        MlpWeightsDev w{};
        layout(w, static_cast<char *>(blob), F, H);
        w.s_out = (float)m->s_out;
        e = cudaMemcpy(w.theta, th.data(), th.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(const_cast<float *>(w.s_in), sin.data(), 256, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = mlp_prepare();
        if (e == cudaSuccess) e = mlp_tile_weights(w, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        count_launches(4);
        if (e != cudaSuccess) {
            cudaFree(blob);
            return cuda_error(e, "scivr_pes_set_mlp: upload");
        }
        void *old = pes->mlp_blob;
        pes->mlp_blob = blob;
        pes->dev.mlp = w;
        if (old) cudaFree(old);
    } else {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_error(e, "scivr_pes_set_mlp: synchronize");
        if (pes->mlp_blob) cudaFree(pes->mlp_blob);
        pes->mlp_blob = nullptr;
        pes->dev.mlp = MlpWeightsDev{};
    }
    clear_error();
    return SCIVR_OK;
}

int scivr_mlp_eval(scivr_pes pes, int64_t n, const float *q, float *V, float *g, float *H, void *stream)
{
    int rc = need_mlp(pes, "scivr_mlp_eval");
    if (rc != SCIVR_OK) return rc;
    if (n < 1) return err(SCIVR_EINVAL, "scivr_mlp_eval: n=%lld < 1", (long long)n);
    if (!q || !V || !g) return err(SCIVR_EINVAL, "scivr_mlp_eval: NULL device pointer");
    const int F = pes->dev.F;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *scr = nullptr;
    cudaError_t e = cudaMallocAsync(&scr, mlp_eval_scratch_bytes(F, n, H != nullptr), s);
    if (e != cudaSuccess) return cuda_error(e, "scivr_mlp_eval: cudaMallocAsync");
    int nl = 0;
    e = mlp_prepare();
    if (e == cudaSuccess) e = mlp_eval(pes->dev.mlp, F, n, q, V, g, H, scr, s, &nl);
    count_launches(nl);
    cudaError_t e2 = cudaFreeAsync(scr, s);
    if (e != cudaSuccess) return cuda_error(e, "scivr_mlp_eval: launch");
    if (e2 != cudaSuccess) return cuda_error(e2, "scivr_mlp_eval: cudaFreeAsync");
    clear_error();
    return SCIVR_OK;
}

int scivr_mlp_get_params(scivr_pes pes, float *theta, void *stream)
{
    int rc = need_mlp(pes, "scivr_mlp_get_params");
    if (rc != SCIVR_OK) return rc;
    if (!theta) return err(SCIVR_EINVAL, "scivr_mlp_get_params: NULL");
    const MlpWeightsDev &w = pes->dev.mlp;
    cudaError_t e = cudaMemcpyAsync(theta, w.theta, (size_t)w.n_params * 4, cudaMemcpyDeviceToDevice,
                                    static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_error(e, "scivr_mlp_get_params: copy");
    clear_error();
    return SCIVR_OK;
}

int scivr_mlp_set_params(scivr_pes pes, const float *theta, void *stream)
{
    int rc = need_mlp(pes, "scivr_mlp_set_params");
    if (rc != SCIVR_OK) return rc;
    if (!theta) return err(SCIVR_EINVAL, "scivr_mlp_set_params: NULL");
    const MlpWeightsDev &w = pes->dev.mlp;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(w.theta, theta, (size_t)w.n_params * 4, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = mlp_tile_weights(w, s);
    count_launches(4);
    if (e != cudaSuccess) return cuda_error(e, "scivr_mlp_set_params");
    clear_error();
    return SCIVR_OK;
}

int scivr_mlp_loss_grad(scivr_pes pes, int64_t n, const float *q, const float *Vref, const float *gref,
                        double alpha, double beta, float *grad, float *loss, void *stream)
{
    int rc = need_mlp(pes, "scivr_mlp_loss_grad");
    if (rc != SCIVR_OK) return rc;
    if (n < 1) return err(SCIVR_EINVAL, "scivr_mlp_loss_grad: n=%lld < 1", (long long)n);
    if (!q || !Vref || !gref || !grad || !loss) return err(SCIVR_EINVAL, "scivr_mlp_loss_grad: NULL device pointer");
    if (!(alpha >= 0.0) || !(beta >= 0.0) || !std::isfinite(alpha) || !std::isfinite(beta))
        return err(SCIVR_EINVAL, "scivr_mlp_loss_grad: alpha and beta must be finite and >= 0");
    const int F = pes->dev.F;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void *scr = nullptr;
    cudaError_t e = cudaMallocAsync(&scr, mlp_train_scratch_bytes(F, n), s);
    if (e != cudaSuccess) return cuda_error(e, "scivr_mlp_loss_grad: cudaMallocAsync");
    int nl = 0;
    e = mlp_prepare();
    if (e == cudaSuccess)
        e = mlp_loss_grad(pes->dev.mlp, F, n, q, Vref, gref, (float)alpha, (float)beta, grad, loss, scr, s, &nl);
    count_launches(nl);
    cudaError_t e2 = cudaFreeAsync(scr, s);
    if (e != cudaSuccess) return cuda_error(e, "scivr_mlp_loss_grad: launch");
    if (e2 != cudaSuccess) return cuda_error(e2, "scivr_mlp_loss_grad: cudaFreeAsync");
    clear_error();
    return SCIVR_OK;
}

int scivr_mlp_adamw(scivr_pes pes, const float *grad, float *m1, float *m2, int32_t t, double lr, double beta1,
                    double beta2, double eps, double weight_decay, void *stream)
{
    int rc = need_mlp(pes, "scivr_mlp_adamw");
    if (rc != SCIVR_OK) return rc;
    if (!grad || !m1 || !m2) return err(SCIVR_EINVAL, "scivr_mlp_adamw: NULL device pointer");
    if (t < 1) return err(SCIVR_EINVAL, "scivr_mlp_adamw: t=%d < 1", t);
    if (!(lr >= 0.0) || !(beta1 >= 0.0 && beta1 < 1.0) || !(beta2 >= 0.0 && beta2 < 1.0) || !(eps > 0.0) ||
        !(weight_decay >= 0.0))
        return err(SCIVR_EINVAL, "scivr_mlp_adamw: hyper-parameters out of range");
    const double c1 = 1.0 - std::pow(beta1, t), c2 = 1.0 - std::pow(beta2, t);
    cudaError_t e = mlp_adamw(pes->dev.mlp, grad, m1, m2, (float)lr, (float)beta1, (float)beta2, (float)eps,
                              (float)weight_decay, (float)c1, (float)c2, static_cast<cudaStream_t>(stream));
    count_launches(5);
    if (e != cudaSuccess) return cuda_error(e, "scivr_mlp_adamw: launch");
    clear_error();
    return SCIVR_OK;
}

int scivr_pes_eval(scivr_pes pes, int64_t n, const double *q, int32_t terms, double *V, double *g, double *H,
                   void *stream)
{
    if (!pes) return err(SCIVR_EINVAL, "scivr_pes_eval: NULL potential");
    if (n < 1) return err(SCIVR_EINVAL, "scivr_pes_eval: n=%lld < 1", (long long)n);
    if (!q || !V) return err(SCIVR_EINVAL, "scivr_pes_eval: NULL device pointer");
    if (terms != SCIVR_TERMS_ALL && terms != SCIVR_TERMS_DIAG && terms != SCIVR_TERMS_COUPLING)
        return err(SCIVR_EINVAL, "scivr_pes_eval: terms=%d invalid", terms);
    if (pes->dev.F > 9) return err(SCIVR_EUNSUPPORTED, "scivr_pes_eval: F=%d > 9 not built", pes->dev.F);
    if (pes->dev.kind == SCIVR_PES_CART3 && terms != SCIVR_TERMS_ALL)
        return err(SCIVR_EINVAL, "scivr_pes_eval: a Cartesian surface has no diagonal/coupling split (terms=%d)", terms);
    cudaError_t e = launch_pes_eval(pes->dev, n, q, terms, V, g, H, static_cast<cudaStream_t>(stream));
    count_launches(1);
    if (e != cudaSuccess) return cuda_error(e, "scivr_pes_eval: launch");
    clear_error();
    return SCIVR_OK;
}

}  // extern "C"
