"""CPU oracle for CDDT ray casting and the beam sensor model.

TEST INFRASTRUCTURE: imported only by the tests, the smoke check and the
benchmark's CPU-baseline leg.  Nothing in the product package imports it.
"""
