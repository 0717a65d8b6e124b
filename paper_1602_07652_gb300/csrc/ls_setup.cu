// ls_setup.cu -- off-line precompute of Sec. 2: quadrature weights and stencils.
//
//  * G_w(d) = h^2 G(h|d|) = h^2 (-i/4) (J_0 + i Y_0)(w h |d|) for d != 0 (trapezoidal
//    rule, Sec. 2, eq. Greens_function), tabulated on [-n, n]^2 on the device.
//  * G_w(0): the diagonal weight.  The paper only says that the rule modifies the
//    diagonal weight and reaches order h^4 log h.  We use the weight that removes
//    the leading defect of the punctured lattice sum of the log singularity:
//        G_w(0) = h^2 [ (log(w h / 2) + gamma + Z'(0) / 2) / (2 pi) - i/4 ],
//    Z'(0) = -log(2 pi) - 2 log(Gamma(1/4)^2 / (2 pi sqrt 2)) (square-lattice Epstein
//    zeta function); with it the rule converges at fourth order.
//  * Sparsifying stencils (Sec. 2): for each of the 9 point types (interior, 4
//    edges, 4 corners) alpha minimises ||alpha G(mu, mu^c)|| over unit vectors.
//    The minimiser is the eigenvector of the smallest eigenvalue of the Gram
//    matrix K = M M^H, M = [G_w(d - p)]_{d in mu, p in window \ mu}; K is summed on
//    the device in FP64 and diagonalised on the host (Jacobi).  alpha = conj(v),
//    scaled so its centre entry is real positive.  The window is every offset of
//    the grid, clipped to the half-plane / quadrant inside Omega for edge and
//    corner types.
//  * beta_d = sum_{e in mu} alpha_e G_w(e - d): the entries of A G kept by the
//    sparsification C = A H on the 9-point pattern (Sec. 2).
#include <cmath>
#include <cstring>
#include <vector>

#include "ls_internal.cuh"

namespace {

__global__ void k_green_table(int n, double h, double omega, double2 w0, double2* gtab) {
    const size_t W = 2 * (size_t)n + 1;
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= W * W) return;
    const int dz = (int)(idx / W) - n, dx = (int)(idx % W) - n;
    if (dx == 0 && dz == 0) {
        gtab[idx] = w0;
        return;
    }
    const double r = h * sqrt((double)dx * dx + (double)dz * dz);
    const double x = omega * r;
    const double J = j0(x), Y = y0(x);
    gtab[idx] = make_double2(0.25 * h * h * Y, -0.25 * h * h * J);
}

struct GramJob {
    int ns;            // stencil points
    int dx[9], dz[9];  // their offsets
    int xlo, xhi, zlo, zhi;
};

// partial[b][a][c] = sum over this block's window points p of G(d_a - p) conj(G(d_c - p))
__global__ void k_gram(int n, GramJob job, const double2* __restrict__ gtab, double2* partial) {
    const int a = blockIdx.y;
    const long long W = 2LL * n + 1;
    const long long nxw = job.xhi - job.xlo + 1;
    const long long cnt = nxw * (job.zhi - job.zlo + 1);
    double2 acc[9];
#pragma unroll
    for (int c = 0; c < 9; ++c) acc[c] = make_double2(0, 0);
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < cnt;
         p += (long long)gridDim.x * blockDim.x) {
        const int px = job.xlo + (int)(p % nxw), pz = job.zlo + (int)(p / nxw);
        if (px >= -1 && px <= 1 && pz >= -1 && pz <= 1) continue;  // p in mu: not in mu^c
        const double2 ga = __ldg(&gtab[(job.dz[a] - pz + n) * W + (job.dx[a] - px + n)]);
#pragma unroll
        for (int c = 0; c < 9; ++c) {
            if (c < job.ns) {
                const double2 gc = __ldg(&gtab[(job.dz[c] - pz + n) * W + (job.dx[c] - px + n)]);
                acc[c] = cconjmul_acc(gc, ga, acc[c]);  // ga * conj(gc)
            }
        }
    }
    __shared__ double2 red[256];
    for (int c = 0; c < job.ns; ++c) {
        red[threadIdx.x] = acc[c];
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[((size_t)blockIdx.x * 9 + a) * 9 + c] = red[0];
        __syncthreads();
    }
}

// Smallest eigenpair of a Hermitian ns x ns matrix via cyclic Jacobi on the real
// symmetric embedding [[Re, -Im], [Im, Re]] (each eigenvalue appears twice).
void hermitian_min_eigvec(int ns, const double2* K, double2* v) {
    const int N = 2 * ns;
    std::vector<double> A(N * N), V(N * N, 0.0);
    for (int r = 0; r < ns; ++r)
        for (int c = 0; c < ns; ++c) {
            const double re = K[r * 9 + c].x, im = K[r * 9 + c].y;
            A[r * N + c] = re;
            A[(r + ns) * N + (c + ns)] = re;
            A[r * N + (c + ns)] = -im;
            A[(r + ns) * N + c] = im;
        }
    for (int i = 0; i < N; ++i) V[i * N + i] = 1.0;
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = 0, diag = 0;
        for (int i = 0; i < N; ++i)
            for (int j = 0; j < N; ++j) (i == j ? diag : off) += A[i * N + j] * A[i * N + j];
        if (off <= 1e-32 * diag) break;
        for (int p = 0; p < N - 1; ++p)
            for (int q = p + 1; q < N; ++q) {
                const double apq = A[p * N + q];
                if (apq == 0.0) continue;
                const double theta = (A[q * N + q] - A[p * N + p]) / (2.0 * apq);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
                for (int k = 0; k < N; ++k) {  // A <- A J (columns p, q)
                    const double akp = A[k * N + p], akq = A[k * N + q];
                    A[k * N + p] = c * akp - s * akq;
                    A[k * N + q] = s * akp + c * akq;
                }
                for (int k = 0; k < N; ++k) {  // A <- J^T A (rows p, q)
                    const double apk = A[p * N + k], aqk = A[q * N + k];
                    A[p * N + k] = c * apk - s * aqk;
                    A[q * N + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < N; ++k) {
                    const double vkp = V[k * N + p], vkq = V[k * N + q];
                    V[k * N + p] = c * vkp - s * vkq;
                    V[k * N + q] = s * vkp + c * vkq;
                }
            }
    }
    int best = 0;
    for (int i = 1; i < N; ++i)
        if (A[i * N + i] < A[best * N + best]) best = i;
    double nrm = 0;
    for (int r = 0; r < ns; ++r) {
        v[r] = make_double2(V[r * N + best], V[(r + ns) * N + best]);
        nrm += v[r].x * v[r].x + v[r].y * v[r].y;
    }
    nrm = std::sqrt(nrm);
    for (int r = 0; r < ns; ++r) v[r] = make_double2(v[r].x / nrm, v[r].y / nrm);
}

int type_index(int bx, int bz) { return (bz + 1) * 3 + (bx + 1); }
int slot_index(int dx, int dz) { return (dz + 1) * 3 + (dx + 1); }

}  // namespace

int ls_green_table(ls_handle* h, double2** gtab_out) {
    const int n = h->n;
    // diagonal weight (Sec. 2; reading in the file header)
    const double kGamma = 0.57721566490153286061;
    const double pi = 3.14159265358979323846;
    const double beta_p0 = std::log(std::tgamma(0.25) * std::tgamma(0.25) / (2.0 * pi * std::sqrt(2.0)));
    const double zeta_p0 = -std::log(2.0 * pi) - 2.0 * beta_p0;
    const double cre = (std::log(h->omega * h->h / 2.0) + kGamma + 0.5 * zeta_p0) / (2.0 * pi);
    h->w0 = make_double2(h->h * h->h * cre, -0.25 * h->h * h->h);
    const size_t W = 2 * (size_t)n + 1;
    double2* g = nullptr;
    LS_CUDA(cudaMalloc(&g, sizeof(double2) * W * W));
    k_green_table<<<(unsigned)((W * W + 255) / 256), 256, 0, h->stream>>>(n, h->h, h->omega, h->w0, g);
    h->launches++;
    cudaError_t e = cudaPeekAtLastError();
    if (e != cudaSuccess) {
        cudaFree(g);
        return ls_cuda_fail(e);
    }
    *gtab_out = g;
    return LS_OK;
}

int ls_stencils_build(ls_handle* h, const double2* gtab) {
    const int n = h->n;
    const int NB = 304;
    double2* partial = nullptr;
    LS_CUDA(cudaMalloc(&partial, sizeof(double2) * NB * 81));
    std::vector<double2> hp(NB * 81);
    // G_w on [-2, 2]^2 for beta
    const size_t W = 2 * (size_t)n + 1;
    double2 gc[5][5];
    int rc = LS_OK;
    for (int dz = -2; dz <= 2 && rc == LS_OK; ++dz) {
        cudaError_t e = cudaMemcpyAsync(gc[dz + 2], gtab + (size_t)(dz + n) * W + (n - 2), sizeof(double2) * 5,
                                        cudaMemcpyDeviceToHost, h->stream);
        if (e != cudaSuccess) rc = ls_cuda_fail(e);
    }
    StencilTables& T = h->tabs[0];
    std::memset(&T, 0, sizeof(T));
    for (int bz = -1; bz <= 1 && rc == LS_OK; ++bz)
        for (int bx = -1; bx <= 1 && rc == LS_OK; ++bx) {
            GramJob job{};
            int slots[9];
            for (int dz = -1; dz <= 1; ++dz)
                for (int dx = -1; dx <= 1; ++dx) {
                    if ((bx == -1 && dx == -1) || (bx == 1 && dx == 1)) continue;
                    if ((bz == -1 && dz == -1) || (bz == 1 && dz == 1)) continue;
                    slots[job.ns] = slot_index(dx, dz);
                    job.dx[job.ns] = dx;
                    job.dz[job.ns] = dz;
                    job.ns++;
                }
            job.xlo = bx == -1 ? 0 : -(n - 1);
            job.xhi = bx == 1 ? 0 : (n - 1);
            job.zlo = bz == -1 ? 0 : -(n - 1);
            job.zhi = bz == 1 ? 0 : (n - 1);
            k_gram<<<dim3(NB, job.ns), 256, 0, h->stream>>>(n, job, gtab, partial);
            h->launches++;
            cudaError_t e = cudaPeekAtLastError();
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(hp.data(), partial, sizeof(double2) * NB * 81, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) {
                rc = ls_cuda_fail(e);
                break;
            }
            double2 K[81];
            for (int a = 0; a < job.ns; ++a)
                for (int c = 0; c < job.ns; ++c) {
                    double2 s = make_double2(0, 0);
                    for (int b = 0; b < NB; ++b) s = s + hp[((size_t)b * 9 + a) * 9 + c];
                    K[a * 9 + c] = s;
                }
            double2 v[9];
            hermitian_min_eigvec(job.ns, K, v);
            // alpha = conj(v), centre real positive
            int ic = 0;
            for (int a = 0; a < job.ns; ++a)
                if (job.dx[a] == 0 && job.dz[a] == 0) ic = a;
            const double2 cc = conj(v[ic]);
            const double ac = std::sqrt(cabs2(cc));
            const double2 ph = make_double2(cc.x / ac, -cc.y / ac);  // conj(cc)/|cc|
            const int t = type_index(bx, bz);
            for (int a = 0; a < job.ns; ++a) T.alpha[t * 9 + slots[a]] = conj(v[a]) * ph;
            // beta_d = sum_e alpha_e G_w(e - d)
            const double w2 = h->omega * h->omega;
            for (int a = 0; a < job.ns; ++a) {
                double2 acc = make_double2(0, 0);
                for (int e2 = 0; e2 < job.ns; ++e2)
                    acc = acc + T.alpha[t * 9 + slots[e2]] * gc[job.dz[e2] - job.dz[a] + 2][job.dx[e2] - job.dx[a] + 2];
                T.wbeta[t * 9 + slots[a]] = w2 * acc;
            }
        }
    cudaFree(partial);
    if (rc != LS_OK) return rc;
    // transposed grid: swap the base-3 digits of type and slot
    StencilTables& TT = h->tabs[1];
    for (int t = 0; t < 9; ++t)
        for (int s = 0; s < 9; ++s) {
            const int tt = (t % 3) * 3 + t / 3, st = (s % 3) * 3 + s / 3;
            TT.alpha[tt * 9 + st] = T.alpha[t * 9 + s];
            TT.wbeta[tt * 9 + st] = T.wbeta[t * 9 + s];
        }
    LS_CUDA(cudaMalloc(&h->dtabs, sizeof(StencilTables) * 2));
    LS_CUDA(cudaMemcpyAsync(h->dtabs, h->tabs, sizeof(StencilTables) * 2, cudaMemcpyHostToDevice, h->stream));
    LS_CUDA(cudaStreamSynchronize(h->stream));
    return LS_OK;
}
