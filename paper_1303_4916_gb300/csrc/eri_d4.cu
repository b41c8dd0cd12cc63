// eri_d4.cu -- kernel instantiations for the classes (dd|ds).
// The classes are spread over several translation units that compile in parallel.
#define HF_COOP_C_dd_ds
#include "eri.cuh"

HF_DEFINE_CLASS_LAUNCHERS(C_dd_ds)

void hf_register_classes_d4(EriClassOps* table) {
  HF_REGISTER_CLASS(table, C_dd_ds, 2, 2, 2, 0, hfgen::C_dd_ds::VRR_FLOPS, hfgen::C_dd_ds::HRR_FLOPS);
}
