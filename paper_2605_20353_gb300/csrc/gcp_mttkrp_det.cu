// gcp_mttkrp_det.cu -- deterministic (sort-by-row) MTTKRP variant.
#include "gcp_internal.h"

gcp_status gcpk_det_grad(gcp_ctx *c, const gcpk::FusedSpec &, int *) {
    c->err = "deterministic MTTKRP not available";
    return GCP_ERR_STATE;
}
