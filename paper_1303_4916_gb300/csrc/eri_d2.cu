// eri_d2.cu -- kernel instantiations for the classes (dp|pp), (dp|ds), (dd|ss), (dd|ps).
// The classes are spread over several translation units that compile in parallel.
#define HF_COOP_C_dp_pp
#define HF_COOP_C_dp_ds
#define HF_COOP_C_dd_ps
#include "eri.cuh"

HF_DEFINE_CLASS_LAUNCHERS(C_dp_pp)
HF_DEFINE_CLASS_LAUNCHERS(C_dp_ds)
HF_DEFINE_CLASS_LAUNCHERS(C_dd_ss)
HF_DEFINE_CLASS_LAUNCHERS(C_dd_ps)

void hf_register_classes_d2(EriClassOps* table) {
  HF_REGISTER_CLASS(table, C_dp_pp, 2, 1, 1, 1, hfgen::C_dp_pp::VRR_FLOPS, hfgen::C_dp_pp::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_dp_ds, 2, 1, 2, 0, hfgen::C_dp_ds::VRR_FLOPS, hfgen::C_dp_ds::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_dd_ss, 2, 2, 0, 0, hfgen::C_dd_ss::VRR_FLOPS, hfgen::C_dd_ss::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_dd_ps, 2, 2, 1, 0, hfgen::C_dd_ps::VRR_FLOPS, hfgen::C_dd_ps::HRR_FLOPS);
}
