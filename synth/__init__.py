"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

Holds workload shapes and random valid surfaces only; none of the model's
update arithmetic lives here.
"""
