// mlp.cu -- the learned planner: a three-layer perceptron that predicts the
// layer latency of a candidate plan from plan and graph statistics, trained
// on measured latencies, and the choice of the candidate it predicts fastest.
//
// y = W3 relu(W2 relu(W1 x + b1) + b2) + b3 in FP32 on CUDA cores (row
// vectors, h = x W + b); mean squared error; gradients layer by layer by the
// chain rule; full-batch Adam (Kingma and Ba, 2015) with bias correction.
// Parameters are packed W1 [in][h], b1 [h], W2 [h][h], b2 [h], W3 [h][1],
// b3 [1].  Every reduction runs in one thread over the batch in order, so
// results are deterministic.  The sizes are tiny (a few thousand rows, 64
// hidden units): the kernels are written for clarity, not speed.
#include <cmath>
#include <vector>

#include "fg_internal.h"

extern std::string g_create_err;

struct fg_mlp {
    int in = 0, h = 0;
    size_t np = 0;
    float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;   // params, grads, Adam moments
    int step = 0;
    // batch buffers
    int cap = 0;
    float *X = nullptr, *y = nullptr, *z1 = nullptr, *a1 = nullptr, *z2 = nullptr, *a2 = nullptr,
          *f = nullptr, *d3 = nullptr, *d2 = nullptr, *d1 = nullptr, *loss = nullptr;
};

namespace {

size_t n_params(int in, int h) { return (size_t)in * h + h + (size_t)h * h + h + h + 1; }

// Z = X W + b (X [n][k], W [k][m]); A = relu(Z) when A is given
__global__ void k_dense(const float *X, const float *W, const float *b, int n, int k, int m, float *Z,
                        float *A)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * m) return;
    const int r = idx / m, c = idx - r * m;
    float s = b[c];
    for (int i = 0; i < k; i++) s += X[(size_t)r * k + i] * W[(size_t)i * m + c];
    Z[idx] = s;
    if (A) A[idx] = s > 0.f ? s : 0.f;
}

// d3 = (2/n)(f - y)
__global__ void k_dout(const float *f, const float *y, int n, float *d3)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r < n) d3[r] = 2.f / (float)n * (f[r] - y[r]);
}

// d[r][i] = (sum_j dn[r][j] W[i][j]) * (z[r][i] > 0);  W [k][m], dn [n][m]
__global__ void k_back(const float *dn, const float *W, const float *z, int n, int k, int m, float *d)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int r = idx / k, i = idx - r * k;
    float s = 0.f;
    for (int j = 0; j < m; j++) s += dn[(size_t)r * m + j] * W[(size_t)i * m + j];
    d[idx] = z[idx] > 0.f ? s : 0.f;
}

// gW[i][j] = sum_r A[r][i] d[r][j] (k*m threads), gb[j] = sum_r d[r][j] (m more)
__global__ void k_gradw(const float *A, const float *d, int n, int k, int m, float *gW, float *gb)
{
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < k * m) {
        const int i = idx / m, j = idx - i * m;
        float s = 0.f;
        for (int r = 0; r < n; r++) s += A[(size_t)r * k + i] * d[(size_t)r * m + j];
        gW[idx] = s;
    } else if (idx < k * m + m) {
        const int j = idx - k * m;
        float s = 0.f;
        for (int r = 0; r < n; r++) s += d[(size_t)r * m + j];
        gb[j] = s;
    }
}

__global__ void k_loss(const float *f, const float *y, int n, float *out)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        float s = 0.f;
        for (int r = 0; r < n; r++) {
            const float e = f[r] - y[r];
            s += e * e;
        }
        *out = s / (float)n;
    }
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, size_t count, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    m[i] = b1 * m[i] + (1.f - b1) * g[i];
    v[i] = b2 * v[i] + (1.f - b2) * g[i] * g[i];
    p[i] -= lr * (m[i] / c1) / (sqrtf(v[i] / c2) + eps);
}

int blocks(size_t n) { return (int)((n + 255) / 256); }

void ensure_batch(fg_mlp *m, int n)
{
    if (n <= m->cap) return;
    float **bufs[] = {&m->X, &m->y, &m->z1, &m->a1, &m->z2, &m->a2, &m->f, &m->d3, &m->d2, &m->d1};
    for (float **b : bufs) {
        cudaFree(*b);
        *b = nullptr;
    }
    const size_t H = (size_t)n * m->h;
    CUDA_TRY(cudaMalloc(&m->X, (size_t)n * m->in * 4));
    CUDA_TRY(cudaMalloc(&m->y, (size_t)n * 4));
    CUDA_TRY(cudaMalloc(&m->z1, H * 4));
    CUDA_TRY(cudaMalloc(&m->a1, H * 4));
    CUDA_TRY(cudaMalloc(&m->z2, H * 4));
    CUDA_TRY(cudaMalloc(&m->a2, H * 4));
    CUDA_TRY(cudaMalloc(&m->f, (size_t)n * 4));
    CUDA_TRY(cudaMalloc(&m->d3, (size_t)n * 4));
    CUDA_TRY(cudaMalloc(&m->d2, H * 4));
    CUDA_TRY(cudaMalloc(&m->d1, H * 4));
    m->cap = n;
}

struct Views {
    float *W1, *b1, *W2, *b2, *W3, *b3;
};

Views views(const fg_mlp *m, float *base)
{
    Views w;
    w.W1 = base;
    w.b1 = w.W1 + (size_t)m->in * m->h;
    w.W2 = w.b1 + m->h;
    w.b2 = w.W2 + (size_t)m->h * m->h;
    w.W3 = w.b2 + m->h;
    w.b3 = w.W3 + m->h;
    return w;
}

void forward(fg_mlp *m, int n)
{
    const Views w = views(m, m->p);
    const int h = m->h;
    k_dense<<<blocks((size_t)n * h), 256>>>(m->X, w.W1, w.b1, n, m->in, h, m->z1, m->a1);
    k_dense<<<blocks((size_t)n * h), 256>>>(m->a1, w.W2, w.b2, n, h, h, m->z2, m->a2);
    k_dense<<<blocks(n), 256>>>(m->a2, w.W3, w.b3, n, h, 1, m->f, nullptr);
    CUDA_TRY(cudaGetLastError());
}

void backward(fg_mlp *m, int n)
{
    const Views w = views(m, m->p), gw = views(m, m->g);
    const int h = m->h;
    k_dout<<<blocks(n), 256>>>(m->f, m->y, n, m->d3);
    k_gradw<<<blocks((size_t)h + 1), 256>>>(m->a2, m->d3, n, h, 1, gw.W3, gw.b3);
    k_back<<<blocks((size_t)n * h), 256>>>(m->d3, w.W3, m->z2, n, h, 1, m->d2);
    k_gradw<<<blocks((size_t)h * h + h), 256>>>(m->a1, m->d2, n, h, h, gw.W2, gw.b2);
    k_back<<<blocks((size_t)n * h), 256>>>(m->d2, w.W2, m->z1, n, h, h, m->d1);
    k_gradw<<<blocks((size_t)m->in * h + h), 256>>>(m->X, m->d1, n, m->in, h, gw.W1, gw.b1);
    CUDA_TRY(cudaGetLastError());
}

void load_batch(fg_mlp *m, const float *X, const float *y, int n)
{
    ensure_batch(m, n);
    CUDA_TRY(cudaMemcpy(m->X, X, (size_t)n * m->in * 4, cudaMemcpyHostToDevice));
    if (y) CUDA_TRY(cudaMemcpy(m->y, y, (size_t)n * 4, cudaMemcpyHostToDevice));
}

#define MLP_TRY try {
#define MLP_CATCH                                                                                  \
    }                                                                                              \
    catch (const fg_error &e) {                                                                    \
        g_create_err = e.what();                                                                   \
        return e.code;                                                                             \
    }                                                                                              \
    catch (const std::exception &e) {                                                              \
        g_create_err = e.what();                                                                   \
        return FG_EOOM;                                                                            \
    }                                                                                              \
    return FG_OK;

}  // namespace

extern "C" {

int fg_mlp_create(int n_in, int hidden, const float *params, fg_mlp **out)
{
    if (!out || !params || n_in < 1 || n_in > 256 || hidden < 1 || hidden > 1024) return FG_EINVAL;
    fg_mlp *m = new fg_mlp;
    MLP_TRY
    m->in = n_in;
    m->h = hidden;
    m->np = n_params(n_in, hidden);
    CUDA_TRY(cudaMalloc(&m->p, m->np * 4));
    CUDA_TRY(cudaMalloc(&m->g, m->np * 4));
    CUDA_TRY(cudaMalloc(&m->m, m->np * 4));
    CUDA_TRY(cudaMalloc(&m->v, m->np * 4));
    CUDA_TRY(cudaMemcpy(m->p, params, m->np * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemset(m->m, 0, m->np * 4));
    CUDA_TRY(cudaMemset(m->v, 0, m->np * 4));
    CUDA_TRY(cudaMalloc(&m->loss, 4));
    *out = m;
    m = nullptr;
    }
    catch (const fg_error &e) {
        g_create_err = e.what();
        fg_mlp_destroy(m);
        return e.code;
    }
    catch (const std::exception &e) {
        g_create_err = e.what();
        fg_mlp_destroy(m);
        return FG_EOOM;
    }
    return FG_OK;
}

int fg_mlp_destroy(fg_mlp *m)
{
    if (!m) return FG_OK;
    float *bufs[] = {m->p, m->g, m->m, m->v, m->X, m->y, m->z1, m->a1, m->z2, m->a2, m->f, m->d3,
                     m->d2, m->d1, m->loss};
    for (float *b : bufs) cudaFree(b);
    delete m;
    return FG_OK;
}

int fg_mlp_params(const fg_mlp *m, float *out)
{
    if (!m || !out) return FG_EINVAL;
    MLP_TRY
    CUDA_TRY(cudaMemcpy(out, m->p, m->np * 4, cudaMemcpyDeviceToHost));
    MLP_CATCH
}

int fg_mlp_forward(fg_mlp *m, const float *X, int n, float *y)
{
    if (!m || !X || !y || n < 1) return FG_EINVAL;
    MLP_TRY
    load_batch(m, X, nullptr, n);
    forward(m, n);
    CUDA_TRY(cudaMemcpy(y, m->f, (size_t)n * 4, cudaMemcpyDeviceToHost));
    MLP_CATCH
}

int fg_mlp_grad(fg_mlp *m, const float *X, const float *y, int n, float *loss, float *grad)
{
    if (!m || !X || !y || n < 1) return FG_EINVAL;
    MLP_TRY
    load_batch(m, X, y, n);
    forward(m, n);
    backward(m, n);
    k_loss<<<1, 32>>>(m->f, m->y, n, m->loss);
    CUDA_TRY(cudaGetLastError());
    if (loss) CUDA_TRY(cudaMemcpy(loss, m->loss, 4, cudaMemcpyDeviceToHost));
    if (grad) CUDA_TRY(cudaMemcpy(grad, m->g, m->np * 4, cudaMemcpyDeviceToHost));
    MLP_CATCH
}

int fg_mlp_train(fg_mlp *m, const float *X, const float *y, int n, int steps, float lr, float *losses)
{
    if (!m || !X || !y || n < 1 || steps < 0 || !(lr > 0)) return FG_EINVAL;
    MLP_TRY
    load_batch(m, X, y, n);
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    std::vector<float> hl(steps);
    float *dl = nullptr;
    if (steps) CUDA_TRY(cudaMalloc(&dl, (size_t)steps * 4));
    for (int s = 0; s < steps; s++) {
        forward(m, n);
        k_loss<<<1, 32>>>(m->f, m->y, n, dl + s);
        backward(m, n);
        m->step++;
        const float c1 = 1.f - std::pow(b1, (float)m->step), c2 = 1.f - std::pow(b2, (float)m->step);
        k_adam<<<blocks(m->np), 256>>>(m->p, m->g, m->m, m->v, m->np, lr, b1, b2, eps, c1, c2);
        CUDA_TRY(cudaGetLastError());
    }
    if (steps) {
        CUDA_TRY(cudaMemcpy(hl.data(), dl, (size_t)steps * 4, cudaMemcpyDeviceToHost));
        cudaFree(dl);
    }
    if (losses)
        for (int s = 0; s < steps; s++) losses[s] = hl[s];
    MLP_CATCH
}

int fg_plan_choose(fg_mlp *m, const float *features, int n_cand, float *pred, int *best)
{
    if (!m || !features || !best || n_cand < 1) return FG_EINVAL;
    std::vector<float> y(n_cand);
    const int rc = fg_mlp_forward(m, features, n_cand, y.data());
    if (rc != FG_OK) return rc;
    int b = 0;
    for (int i = 1; i < n_cand; i++)
        if (y[i] < y[b]) b = i;
    *best = b;
    if (pred)
        for (int i = 0; i < n_cand; i++) pred[i] = y[i];
    return FG_OK;
}

}  // extern "C"
