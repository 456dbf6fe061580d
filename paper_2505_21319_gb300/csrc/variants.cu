// Dispatch of the ablation-variant kernels by value degree.
#include "variants.cuh"

namespace efunc {
namespace variant {

int sm_count() { return device_sm_count(); }

}  // namespace variant

int variant_key_records(int sets, int deg) { return variant::nsets_of(sets) * variant::nrec_of(deg); }

cudaError_t launch_variant_pack(const VariantArgs &a, cudaStream_t s)
{
    switch (a.deg) {
    case 0: return variant::launch_pack_deg0(a, s);
    case 1: return variant::launch_pack_deg1(a, s);
    case 2: return variant::launch_pack_deg2(a, s);
    default: return variant::launch_pack_deg3(a, s);
    }
}

cudaError_t launch_variant(const VariantArgs &a, int mode, cudaStream_t s)
{
    switch (a.deg) {
    case 0: return variant::launch_deg0(a, mode, s);
    case 1: return variant::launch_deg1(a, mode, s);
    case 2: return variant::launch_deg2(a, mode, s);
    default: return variant::launch_deg3(a, mode, s);
    }
}

}  // namespace efunc
