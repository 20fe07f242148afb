"""FP64 CPU oracle of the SIPF-PIC step.

Test infrastructure only: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the library.
"""
