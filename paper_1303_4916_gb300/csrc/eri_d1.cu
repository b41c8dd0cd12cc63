// eri_d1.cu -- kernel instantiations for the classes (ds|ss), (ds|ps), (ds|pp), (ds|ds), (dp|ss), (dp|ps).
// The classes are spread over several translation units that compile in parallel.
#include "eri.cuh"

HF_DEFINE_CLASS_LAUNCHERS(C_ds_ss)
HF_DEFINE_CLASS_LAUNCHERS(C_ds_ps)
HF_DEFINE_CLASS_LAUNCHERS(C_ds_pp)
HF_DEFINE_CLASS_LAUNCHERS(C_ds_ds)
HF_DEFINE_CLASS_LAUNCHERS(C_dp_ss)
HF_DEFINE_CLASS_LAUNCHERS(C_dp_ps)

void hf_register_classes_d1(EriClassOps* table) {
  HF_REGISTER_CLASS(table, C_ds_ss, 2, 0, 0, 0, hfgen::C_ds_ss::VRR_FLOPS, hfgen::C_ds_ss::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_ds_ps, 2, 0, 1, 0, hfgen::C_ds_ps::VRR_FLOPS, hfgen::C_ds_ps::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_ds_pp, 2, 0, 1, 1, hfgen::C_ds_pp::VRR_FLOPS, hfgen::C_ds_pp::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_ds_ds, 2, 0, 2, 0, hfgen::C_ds_ds::VRR_FLOPS, hfgen::C_ds_ds::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_dp_ss, 2, 1, 0, 0, hfgen::C_dp_ss::VRR_FLOPS, hfgen::C_dp_ss::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_dp_ps, 2, 1, 1, 0, hfgen::C_dp_ps::VRR_FLOPS, hfgen::C_dp_ps::HRR_FLOPS);
}
