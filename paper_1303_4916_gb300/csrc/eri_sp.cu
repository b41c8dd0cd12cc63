// eri_sp.cu -- kernel instantiations for the classes (ss|ss), (ps|ss), (ps|ps), (pp|ss), (pp|ps), (pp|pp).
// The classes are spread over several translation units that compile in parallel.
#include "eri.cuh"

HF_DEFINE_CLASS_LAUNCHERS(C_ss_ss)
HF_DEFINE_CLASS_LAUNCHERS(C_ps_ss)
HF_DEFINE_CLASS_LAUNCHERS(C_ps_ps)
HF_DEFINE_CLASS_LAUNCHERS(C_pp_ss)
HF_DEFINE_CLASS_LAUNCHERS(C_pp_ps)
HF_DEFINE_CLASS_LAUNCHERS(C_pp_pp)

void hf_register_classes_sp(EriClassOps* table) {
  HF_REGISTER_CLASS(table, C_ss_ss, 0, 0, 0, 0, hfgen::C_ss_ss::VRR_FLOPS, hfgen::C_ss_ss::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_ps_ss, 1, 0, 0, 0, hfgen::C_ps_ss::VRR_FLOPS, hfgen::C_ps_ss::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_ps_ps, 1, 0, 1, 0, hfgen::C_ps_ps::VRR_FLOPS, hfgen::C_ps_ps::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_pp_ss, 1, 1, 0, 0, hfgen::C_pp_ss::VRR_FLOPS, hfgen::C_pp_ss::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_pp_ps, 1, 1, 1, 0, hfgen::C_pp_ps::VRR_FLOPS, hfgen::C_pp_ps::HRR_FLOPS);
  HF_REGISTER_CLASS(table, C_pp_pp, 1, 1, 1, 1, hfgen::C_pp_pp::VRR_FLOPS, hfgen::C_pp_pp::HRR_FLOPS);
}
