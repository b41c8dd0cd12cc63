// eri_d5.cu -- kernel instantiations for the classes (dd|dp).
// The classes are spread over several translation units that compile in parallel.
#define HF_COOP_C_dd_dp
#include "eri.cuh"

HF_DEFINE_CLASS_LAUNCHERS(C_dd_dp)

void hf_register_classes_d5(EriClassOps* table) {
  HF_REGISTER_CLASS(table, C_dd_dp, 2, 2, 2, 1, hfgen::C_dd_dp::VRR_FLOPS, hfgen::C_dd_dp::HRR_FLOPS);
}
