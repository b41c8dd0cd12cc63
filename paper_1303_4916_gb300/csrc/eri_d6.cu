// eri_d6.cu -- kernel instantiations for the classes (dd|dd).
// The classes are spread over several translation units that compile in parallel.
#define HF_COOP_C_dd_dd
#include "eri.cuh"

HF_DEFINE_CLASS_LAUNCHERS(C_dd_dd)

void hf_register_classes_d6(EriClassOps* table) {
  HF_REGISTER_CLASS(table, C_dd_dd, 2, 2, 2, 2, hfgen::C_dd_dd::VRR_FLOPS, hfgen::C_dd_dd::HRR_FLOPS);
}
