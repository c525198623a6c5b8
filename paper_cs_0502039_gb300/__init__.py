"""GB300-native exact simulator of Poisson-asynchronous cellular arrays.

Glauber's continuous-time Ising model on a periodic 2D lattice, simulated
exactly in parallel after Lubachevsky, "Efficient Parallel Simulations of
Asynchronous Cellular Arrays".  The compute path is the hand-written sm_103a
CUDA library ``libac.so`` behind the C ABI of ``include/ac.h``; :mod:`.ac` is
its thin ctypes binding.
"""
from .ac import (AC_INIT_DOWN, AC_INIT_RANDOM, AC_INIT_UP, AC_KERNEL_BLOCKED, AC_KERNEL_EPOCH, AC_KERNEL_ROUND,  # noqa: F401
                 AC_LAW_EXP, AC_LAW_ROOT8, AC_LAW_UNIFORM, AC_LIFE_CONWAY_BIRTH, AC_LIFE_CONWAY_SURVIVE,
                 AC_MAX_FRAMES, AC_RATE_ONE, AC_OPT_DROP_PUBLISH, AC_OPT_EARLY_REJECT, AC_OPT_MAX_ROUNDS, AC_OPT_WATCHDOG_NS, TICKS_PER_UNIT,
                 ACError, Sim, ac_batch_create, ac_class_counts, ac_create_life, ac_create_q, ising_q, life, ac_batch_run_until, ac_configure, ac_create, ac_destroy,
                 ac_dev_exp_ticks, ac_dev_philox, ac_frames_configure, ac_frames_status, ac_load_state, ac_load_state_async,
                 ac_read_state, ac_read_state_async, ac_read_state_device, ac_reset, ac_round_history, ac_run_blocked_static,
                 ac_run_until, ac_run_until_frames, ac_run_until_ticks, ac_set_option, ac_set_rates, ac_set_stream, ac_slab_configure,
                 ac_slab_export, ac_slab_import, ac_slab_step, ac_stats,
                 ac_thresholds, ac_time_model)
