// batched_f64.cu -- the batched solver's plans with double inner storage, in a
// translation unit of their own so that the three storages compile in parallel.
#include "batched_impl.cuh"

namespace stag {

int batched_run_f64(stag_ctx ctx, BatchSlot& m, int recon, const void* lk, const double2* x0, double mass,
                    const double* shifts_dev, const stag_solver_params& prm, double delta, int nb)
{
    if (recon == 18)
        return run_with_nb<SpinorF64, SpinorF64, LinkField<double2, 18>>(ctx, m, lk, x0, mass, shifts_dev, prm, delta, nb);
    return run_with_nb<SpinorF64, SpinorF64, LinkField<double2, 12>>(ctx, m, lk, x0, mass, shifts_dev, prm, delta, nb);
}

}  // namespace stag
