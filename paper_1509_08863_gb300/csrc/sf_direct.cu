// Instances of the unstaged sweep kernel (cheb_step_direct_kernel), kept in
// their own translation unit so that they compile in parallel with the
// staged ones.
#include "sf_step.cuh"

namespace sf {

template <typename TS, int LPR, bool W>
static StepFn direct_fn(int mode) {
    switch (mode) {
        case MODE_FWD: return cheb_step_direct_kernel<TS, LPR, MODE_FWD, W>;
        case MODE_MOM: return cheb_step_direct_kernel<TS, LPR, MODE_MOM, W>;
        default: return cheb_step_direct_kernel<TS, LPR, MODE_CLEN, W>;
    }
}

template <typename TS, bool W>
static StepFn direct_fn_lpr(int lpr, int mode) {
    switch (lpr) {
        case 2: return direct_fn<TS, 2, W>(mode);
        case 4: return direct_fn<TS, 4, W>(mode);
        case 8: return direct_fn<TS, 8, W>(mode);
        case 16: return direct_fn<TS, 16, W>(mode);
        case 32: return direct_fn<TS, 32, W>(mode);
        default: return nullptr;
    }
}

StepFn direct_step_fn(int storage, int lpr, int mode, bool weighted) {
    if (storage == SF_F32)
        return weighted ? direct_fn_lpr<float, true>(lpr, mode) : direct_fn_lpr<float, false>(lpr, mode);
    if (storage == SF_BF16)
        return weighted ? direct_fn_lpr<__nv_bfloat16, true>(lpr, mode)
                        : direct_fn_lpr<__nv_bfloat16, false>(lpr, mode);
    if (storage == SF_F16)
        return weighted ? direct_fn_lpr<__half, true>(lpr, mode) : direct_fn_lpr<__half, false>(lpr, mode);
    return nullptr;
}

}  // namespace sf
