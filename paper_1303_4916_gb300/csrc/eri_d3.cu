// eri_d3.cu -- kernel instantiations for the classes (dp|dp), (dd|pp).
// The classes are spread over several translation units that compile in parallel.
#define HF_COOP_C_dp_dp
#define HF_COOP_C_dd_pp
#include "eri.cuh"

HF_DEFINE_CLASS_LAUNCHERS(C_dp_dp)
HF_DEFINE_CLASS_LAUNCHERS(C_dd_pp)

void hf_register_classes_d3(EriClassOps* table) {
  HF_REGISTER_CLASS(table, C_dp_dp, 2, 1, 2, 1, hfgen::C_dp_dp::VRR_FLOPS, hfgen::C_dp_dp::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_dd_pp, 2, 2, 1, 1, hfgen::C_dd_pp::VRR_FLOPS, hfgen::C_dd_pp::HRR_FLOPS);
}
