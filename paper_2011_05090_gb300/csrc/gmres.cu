// RGS-Arnoldi (Alg. 3), randomized GMRES (Sec. 4.2) and the CGS2-GMRES comparator.
#include "common.cuh"

extern "C" {

rgs_status rgs_arnoldi_create(rgs_handle, rgs_sketch, int64_t, int32_t, rgs_dtype, rgs_arnoldi* out) {
    if (out) *out = nullptr;
    return RGS_ERR_NOT_IMPLEMENTED;
}
rgs_status rgs_arnoldi_destroy(rgs_arnoldi) { return RGS_ERR_NOT_IMPLEMENTED; }
rgs_status rgs_arnoldi_start(rgs_handle, rgs_arnoldi, const double*) { return RGS_ERR_NOT_IMPLEMENTED; }
rgs_status rgs_arnoldi_step(rgs_handle, rgs_arnoldi, const rgs_csr*, const double*) { return RGS_ERR_NOT_IMPLEMENTED; }
rgs_status rgs_arnoldi_get(rgs_handle, rgs_arnoldi, int32_t*, double*, int64_t, double*) { return RGS_ERR_NOT_IMPLEMENTED; }
rgs_status rgs_arnoldi_basis(rgs_arnoldi, void**, int64_t*) { return RGS_ERR_NOT_IMPLEMENTED; }
rgs_status rgmres_solve(rgs_handle, rgs_sketch, const rgs_csr*, const double*, double*, const rgmres_opts*,
                        rgmres_info*) {
    return RGS_ERR_NOT_IMPLEMENTED;
}
rgs_status cgs2_gmres_solve(rgs_handle, const rgs_csr*, const double*, double*, const rgmres_opts*, rgmres_info*) {
    return RGS_ERR_NOT_IMPLEMENTED;
}
rgs_status rgmres_set_preconditioner(rgs_handle, rgs_precond_kind, const void*, int32_t) {
    return RGS_ERR_NOT_IMPLEMENTED;
}
rgs_status rgmres_solve_batched(rgs_handle, int32_t, const rgs_sketch*, const rgs_csr*, const double* const*,
                                double* const*, const rgmres_opts*, rgmres_info*) {
    return RGS_ERR_NOT_IMPLEMENTED;
}

}  // extern "C"
