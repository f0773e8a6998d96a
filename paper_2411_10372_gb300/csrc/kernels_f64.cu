// FP64 instantiation of the kernels.  Compiled with --fmad=false so that each
// FP64 operation rounds exactly as written (the FP64 path is the one checked
// against the CPU oracle at 1e-12).
#define CM_DEFINE_DIAG_FINAL
#include "kernels_impl.cuh"

namespace cm {

template struct Launch<double>;

bool pdl_enabled()
{
    static int on = -1;
    if (on < 0) {
        const char* e = getenv("CM_PDL");
        on = (e && e[0] == '0') ? 0 : 1;
    }
    return on == 1;
}

cudaError_t launch_diag_final(const double* scratch, const double* zt, const DiagFinal& F, DevCtl* ctl, cm_diag* rec,
                              cudaStream_t s)
{
    diag_final<<<1, kDiagThreads, 0, s>>>(scratch, zt, F, ctl, rec);
    return cudaGetLastError();
}

}  // namespace cm
