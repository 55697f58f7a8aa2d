// Self-consistent-field driver (paper Eq. 2): placeholder entry points until the device SCF lands.
#include "mess_internal.h"

extern "C" mess_status mess_scf(const mess_basis* b, const mess_scf_opts* opts, mess_scf_result* res, double* D_out)
{
    (void)b; (void)opts; (void)res; (void)D_out;
    mess_set_error("mess_scf: not implemented yet");
    return MESS_ENOTIMPL;
}

extern "C" mess_status mess_scf_batch(int nmol, mess_basis* const* bases, const mess_scf_opts* opts, mess_scf_result* res)
{
    (void)nmol; (void)bases; (void)opts; (void)res;
    mess_set_error("mess_scf_batch: not implemented yet");
    return MESS_ENOTIMPL;
}
