// K2: tensor-core form of the fused domain-selection step (placeholder until
// the tcgen05 kernel lands).
#include "ds_internal.cuh"

namespace ising {

int tc_setup(ising_ds* ds) {
  return fail(ds->ctx, ISING_ENOTSUP, "tensor-core path not built yet");
}
int tc_step(ising_ds* ds, bool) { return fail(ds->ctx, ISING_ENOTSUP, "tensor-core path not built yet"); }
void tc_release(ising_ds*) {}

}  // namespace ising
