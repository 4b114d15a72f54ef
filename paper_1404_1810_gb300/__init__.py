"""GB300-native AM-QFT: batched power-of-two complex DFT by the AM-QFT
recursion ("A class of AM-QFT algorithms for power-of-two FFT", Pasquini),
computed by hand-written sm_103a CUDA kernels behind a C ABI (include/amqft.h).
"""
from .amqft import (AMQFT_C64, AMQFT_CBF16, AMQFT_CF16, AMQFT_CI16, AMQFT_CONST_FLY, AMQFT_CONST_TABLE, AmqftError, Plan, RaggedPlan, amqft_destroy,  # noqa: F401
                    amqft_exec_fwd, amqft_exec_host, amqft_exec_inv, amqft_exec_rdft, amqft_exec_irdft, amqft_exec_dct_dst,
                    amqft_exec_ragged, amqft_exec_static, amqft_last_error,
                    amqft_plan_ragged, amqft_ragged_skipped, amqft_ragged_tune, amqft_plan, amqft_plan_info, amqft_plan_launches,
                    amqft_plan_get_constants, amqft_plan_set_constants,
                    amqft_version, dequantize, fft, load)
from .autograd import amqft as amqft_autograd, clear_plan_cache  # noqa: F401,E402
