// C ABI: basis extraction and the online solve.
#include "internal.h"


using namespace msp;

extern "C" msp_status msp_extract_basis(msp_medium m, double tau, int precision, void* stream, msp_basis* out) {
    clear_error();
    MSP_CHECK_ARG(m && out, "msp_extract_basis: NULL argument");
    MSP_CHECK_ARG(tau >= 0 && tau < 1, "msp_extract_basis: tau must lie in [0, 1)");
    MSP_CHECK_ARG(precision == MSP_FP64 || precision == MSP_MIXED, "msp_extract_basis: unknown precision");
    *out = nullptr;
    if (!m->M.sampled) {
        set_error("msp_extract_basis: call msp_sample_patches first");
        return MSP_ERR_STATE;
    }
    auto* b = new msp_basis_s();
    msp_status st = build_basis(m->M, tau, precision, (cudaStream_t)stream, b->B);
    if (st != MSP_OK) {
        delete b;
        return st;
    }
    *out = b;
    return MSP_OK;
}

extern "C" void msp_basis_destroy(msp_basis b) { delete b; }

extern "C" msp_status msp_basis_info(msp_basis b, int patch, int* k, double* sigma_host) {
    clear_error();
    MSP_CHECK_ARG(b, "msp_basis_info: NULL basis");
    MSP_CHECK_ARG(patch >= 0 && patch < (int)b->B.patches.size(), "msp_basis_info: patch out of range");
    if (k) *k = b->B.k[patch];
    if (sigma_host) {
        const int c = b->B.patches[patch].cols;
        for (int i = 0; i < c; ++i) sigma_host[i] = b->B.sigma[b->B.sigma_off[patch] + i];
    }
    return MSP_OK;
}

extern "C" msp_status msp_get_basis(msp_basis b, int patch, double* dst, void* stream) {
    clear_error();
    MSP_CHECK_ARG(b && dst, "msp_get_basis: NULL argument");
    MSP_CHECK_ARG(patch >= 0 && patch < (int)b->B.patches.size(), "msp_get_basis: patch out of range");
    const size_t n = (size_t)b->B.patches[patch].n_k * b->B.k[patch];
    if (n) MSP_CUDA(cudaMemcpyAsync(dst, b->B.Q.p + b->B.q_off[patch], n * sizeof(double), cudaMemcpyDeviceToDevice,
                                    (cudaStream_t)stream));
    return MSP_OK;
}

extern "C" msp_status msp_online_counts(msp_basis b, int* n_unknowns, int* n_rows) {
    clear_error();
    MSP_CHECK_ARG(b, "msp_online_counts: NULL basis");
    if (n_unknowns) *n_unknowns = b->B.Np;
    if (n_rows) *n_rows = b->B.n_rows;
    return MSP_OK;
}

extern "C" msp_status msp_basis_extract_timing(msp_basis b, double* ms_host, double* jacobi_flop_host) {
    clear_error();
    MSP_CHECK_ARG(b && ms_host, "msp_basis_extract_timing: NULL argument");
    const Basis& B = b->B;
    for (int p = 0; p < 6; ++p) ms_host[p] = 0.0;
    if (B.ext_ev.size() == 7) {
        MSP_CUDA(cudaEventSynchronize(B.ext_ev[6]));
        for (int p = 0; p < 6; ++p) {
            float t = 0.f;
            MSP_CUDA(cudaEventElapsedTime(&t, B.ext_ev[p], B.ext_ev[p + 1]));
            ms_host[p] = t;
        }
    }
    if (jacobi_flop_host) {
        // per column pair and sweep: three inner products (3c multiply-adds) and the
        // rotation of the pair's columns of W and of V (4c + 4c): 22c flop
        double f = 0.0;
        for (size_t m = 0; m < B.jac_cols.size() && m < B.jac_sweeps.size(); ++m) {
            const double c = B.jac_cols[m];
            f += (double)B.jac_sweeps[m] * 0.5 * c * (c - 1.0) * 22.0 * c;
        }
        *jacobi_flop_host = f;
    }
    return MSP_OK;
}

extern "C" msp_status msp_online_solve(msp_basis b, const double* phi, int batch, double tol, int max_iter, double* u,
                                       double* c_dev, int* iters_host, void* stream) {
    clear_error();
    MSP_CHECK_ARG(b && phi && (u || c_dev), "msp_online_solve: NULL argument");
    MSP_CHECK_ARG(batch >= 0, "msp_online_solve: negative batch");
    MSP_CHECK_ARG(tol > 0 && tol < 1, "msp_online_solve: tol must lie in (0, 1)");
    MSP_CHECK_ARG(max_iter >= 1, "msp_online_solve: max_iter must be >= 1");
    if (batch == 0) return MSP_OK;
    return online_solve(b->B, phi, batch, tol, max_iter, u, c_dev, iters_host, (cudaStream_t)stream);
}

extern "C" msp_status msp_online_solve_constrained(msp_basis b, const double* phi, int batch, double tol, int max_iter,
                                                   double* u, double* c_dev, int* iters_host, void* stream) {
    clear_error();
    MSP_CHECK_ARG(b && phi && (u || c_dev), "msp_online_solve_constrained: NULL argument");
    MSP_CHECK_ARG(batch >= 0, "msp_online_solve_constrained: negative batch");
    MSP_CHECK_ARG(tol > 0 && tol < 1, "msp_online_solve_constrained: tol must lie in (0, 1)");
    MSP_CHECK_ARG(max_iter >= 1, "msp_online_solve_constrained: max_iter must be >= 1");
    if (batch == 0) return MSP_OK;
    return online_solve_constrained(b->B, phi, batch, tol, max_iter, u, c_dev, iters_host, (cudaStream_t)stream);
}

extern "C" msp_status msp_ras_setup(msp_basis b, msp_medium full, int coarse, void* stream) {
    clear_error();
    MSP_CHECK_ARG(b && full, "msp_ras_setup: NULL argument");
    return ras_setup(b->B, full->M, coarse != 0, (cudaStream_t)stream);
}

extern "C" msp_status msp_online_solve_ras(msp_basis b, const double* phi, int batch, double tol, int max_iter,
                                           double* u, double* c_dev, int* iters_host, void* stream) {
    clear_error();
    MSP_CHECK_ARG(b && phi && (u || c_dev), "msp_online_solve_ras: NULL argument");
    MSP_CHECK_ARG(batch >= 0, "msp_online_solve_ras: negative batch");
    MSP_CHECK_ARG(tol > 0 && tol < 1, "msp_online_solve_ras: tol must lie in (0, 1)");
    MSP_CHECK_ARG(max_iter >= 1, "msp_online_solve_ras: max_iter must be >= 1");
    if (batch == 0) return MSP_OK;
    return ras_solve(b->B, phi, batch, tol, max_iter, u, c_dev, iters_host, (cudaStream_t)stream);
}

extern "C" msp_status msp_basis_build_map(msp_basis b, double tol, int max_iter, void* stream) {
    clear_error();
    MSP_CHECK_ARG(b, "msp_basis_build_map: NULL basis");
    MSP_CHECK_ARG(tol > 0 && tol < 1, "msp_basis_build_map: tol must lie in (0, 1)");
    MSP_CHECK_ARG(max_iter >= 1, "msp_basis_build_map: max_iter must be >= 1");
    return build_online_map(b->B, tol, max_iter, (cudaStream_t)stream);
}

extern "C" msp_status msp_basis_set_map_engine(msp_basis b, int engine) {
    clear_error();
    MSP_CHECK_ARG(b, "msp_basis_set_map_engine: NULL basis");
    MSP_CHECK_ARG(engine == MSP_MAP_TENSOR_CORES || engine == MSP_MAP_CUDA_CORES, "msp_basis_set_map_engine: unknown engine");
    b->B.map_engine = engine;
    return MSP_OK;
}

extern "C" msp_status msp_online_solve_map(msp_basis b, const double* phi, int batch, double* u, void* stream) {
    clear_error();
    MSP_CHECK_ARG(b && phi && u, "msp_online_solve_map: NULL argument");
    MSP_CHECK_ARG(batch >= 0, "msp_online_solve_map: negative batch");
    if (batch == 0) return MSP_OK;
    return online_solve_map(b->B, phi, batch, u, (cudaStream_t)stream, nullptr);
}

extern "C" msp_status msp_basis_get_stats(msp_basis b, msp_basis_stats* out) {
    clear_error();
    MSP_CHECK_ARG(b && out, "msp_basis_get_stats: NULL argument");
    out->max_jacobi_sweeps = b->B.max_jacobi_sweeps;
    out->max_cholqr_tries = b->B.max_cholqr_tries;
    out->online_shift = b->B.bt_shift;
    out->online_blocks = b->B.bt_q;
    out->mean_jacobi_sweeps = b->B.mean_jacobi_sweeps;
    out->online_apply_bits = b->B.use_block_jacobi ? 0
                             : (b->B.bt_prec == 1 ? 32
                                                  : (b->B.bt_prec == 2 ? (b->B.bt_apply_mode == 1 ? 64
                                                                          : b->B.bt_apply_mode == 2 ? 32 : 0)
                                                                       : 0));
    out->online_factor_bits = b->B.use_block_jacobi ? 0 : (b->B.bt_prec == 2 ? 64 : (b->B.bt_prec == 1 ? 32 : 0));
    return MSP_OK;
}

extern "C" msp_status msp_basis_set_preconditioner(msp_basis b, int kind) {
    clear_error();
    MSP_CHECK_ARG(b, "msp_basis_set_preconditioner: NULL basis");
    MSP_CHECK_ARG(kind == MSP_PRECOND_BLOCK_ROWS || kind == MSP_PRECOND_PATCH_BLOCKS ||
                      kind == MSP_PRECOND_BLOCK_ROWS_FP64 || kind == MSP_PRECOND_BLOCK_ROWS_FP32,
                  "msp_basis_set_preconditioner: unknown preconditioner");
    b->B.use_block_jacobi = (kind == MSP_PRECOND_PATCH_BLOCKS);
    b->B.bt_apply_mode = kind == MSP_PRECOND_BLOCK_ROWS_FP64 ? 1 : (kind == MSP_PRECOND_BLOCK_ROWS_FP32 ? 2 : 0);
    return MSP_OK;
}
